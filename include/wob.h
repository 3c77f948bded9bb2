/*
 * wob.h -- C ABI of the GB300 walk-on-boundary (WoB) library.
 *
 * The library estimates solutions of Laplace boundary value problems on
 * closed triangle meshes with the walk-on-boundary method of Sugimoto et al.,
 * "A Practical Walk-on-Boundary Method for Boundary Value Problems"
 * (SIGGRAPH 2023).  Every step of the estimator runs in the library's own
 * CUDA kernels for sm_103a; this header uses plain pointers and sizes only.
 *
 * Conventions for every function:
 *  - The return value is a status: WOB_OK (0) or a negative WOB_ERR_* code.
 *    wob_last_error() returns a message for the calling thread's last error.
 *    No C++ exception crosses this interface.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls enqueue work on it and return without synchronising,
 *    except where noted ("synchronises").
 *  - "device" pointers are CUDA device memory (for example a torch tensor's
 *    data_ptr()); "host" pointers are ordinary host memory.  The library
 *    never frees or keeps memory it did not allocate.
 *  - Meshes: vertices float32 V x 3 (row-major), triangles int32 T x 3,
 *    counter-clockwise when seen from outside the interior domain Omega, so
 *    that (v1 - v0) x (v2 - v0) points out of Omega (the paper keeps normals
 *    oriented outward from Omega for both interior and exterior problems,
 *    Sec. 4.5.1).  The surface must be closed.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *    (seed_lo ^ problem, seed_hi) and counter (query, walk,
 *    step << 16 | purpose << 12 | attempt, extra); results are a
 *    deterministic function of (inputs, seed, walk range) and do not depend
 *    on launch configuration.
 */
#ifndef WOB_H
#define WOB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WOB_OK 0
#define WOB_ERR_INVALID_ARG (-1)     /* bad pointer, size or enum value */
#define WOB_ERR_CUDA (-2)            /* a CUDA runtime call failed */
#define WOB_ERR_OOM (-3)             /* device allocation failed */
#define WOB_ERR_TIMEOUT (-4)         /* a bounded device-side wait gave up */
#define WOB_ERR_DEGENERATE_MESH (-5) /* non-finite vertex, bad index, zero-area
                                        triangle or inward orientation */
#define WOB_ERR_UNSUPPORTED (-6)     /* combination not implemented */
#define WOB_ERR_DEVICE_CHECK (-7)    /* a device-side check fired (traversal
                                        stack overflow or iteration bound);
                                        returned by calls that read the check
                                        back (wob_solve_counted); in every
                                        solve the estimates of a call in
                                        which a check fired are NaN */

/* Boundary-integral formulation (Table 1 of the paper). */
typedef enum {
    WOB_DIRICHLET_DL = 0,   /* Dirichlet data, double-layer potential (Sec. 4.1) */
    WOB_NEUMANN_SL = 1,     /* Neumann data, single-layer potential (Sec. 4.3) */
    WOB_ROBIN_SL = 2,       /* Robin data, single-layer potential (Sec. 4.3) */
    WOB_NEUMANN_DIRECT = 3, /* Neumann data, direct boundary integral equation
                               (Sec. 4.2): lines for the dG/dn_y term, one
                               area-uniform point per vertex for the G q term */
    WOB_MIXED_SL = 4        /* a Dirichlet, Neumann or Robin condition per
                               triangle (bc_type), single-layer potential;
                               Dirichlet parts through mu = mu - k S mu + k u_D
                               sampled with the branch probability p_k (Sec. 4.3) */
} wob_kind;

/* Boundary condition of a triangle in WOB_MIXED_SL problems. */
typedef enum { WOB_BC_DIRICHLET = 0, WOB_BC_NEUMANN = 1, WOB_BC_ROBIN = 2 } wob_bc;

/* How the boundary data is given. */
typedef enum {
    WOB_DATA_VERTEX_P1 = 0, /* per-vertex values, linear over each triangle */
    WOB_DATA_POLY = 1,      /* field h = c0 + c.x + quadratic terms (poly[10]) */
    WOB_DATA_POINT = 2      /* field h = scale / |x - x0| */
} wob_data_mode;

typedef struct wob_mesh_s *wob_mesh;
typedef struct wob_bvh_s *wob_bvh;

typedef struct {
    int64_t V, T;
    double bbox_lo[3], bbox_hi[3];
    double L;        /* bounding-box diagonal */
    double area;     /* total surface area |Gamma| */
    double volume;   /* signed enclosed volume (> 0 for outward orientation) */
    double max_edge; /* longest triangle edge */
} wob_mesh_info;

typedef struct {
    int32_t leaf_size; /* max triangles per leaf, 1..8 (0 = default 1) */
    int32_t reserved[7];
} wob_bvh_params;

typedef struct {
    int64_t nodes;   /* 8-wide nodes */
    int64_t leaves;  /* leaves (triangle groups of at most leaf_size) */
    int32_t depth;   /* depth of the 8-wide tree (root = 0) */
    int32_t leaf_size;
    int64_t bytes;   /* device bytes of the wide nodes + leaf triangles */
} wob_bvh_info;

/*
 * One boundary value problem.
 *   kind/side: formulation and phi = +1 (interior) or -1 (exterior), Table 1.
 *   alpha:     Robin coefficient (WOB_ROBIN_SL), Eq. (PoissonBC).
 *   data:      Dirichlet data g (DL), Neumann flux dh/dn (NEUMANN_SL) or Robin
 *              data dh/dn + alpha h (ROBIN_SL).  In the POLY and POINT modes
 *              the library evaluates these from the harmonic field h; in the
 *              VERTEX_P1 mode vertex_data (device, V floats) is the data itself.
 *   poly:      coefficients of 1, x, y, z, x^2, y^2, z^2, xy, yz, zx.
 *   problem:   stream index folded into the generator key.
 *   tau:       near-degenerate line threshold relative to the mesh diagonal
 *              (0 = default 2e-6); lines passing closer than tau*L to a
 *              triangle edge are flagged in the debug outputs.
 *   bc_type:   WOB_MIXED_SL only: device, T bytes (wob_bc, original triangle
 *              order); data from the field h: u_D = h, q = dh/dn, Robin
 *              dh/dn + alpha h (POLY or POINT mode).
 *   k_mix, p_k: WOB_MIXED_SL only: the constant k > 0 of the Dirichlet parts
 *              and the probability 0 < p_k < 1 of moving (the paper uses 4
 *              and 2/3; on the unit sphere the series converges for k < 2).
 *   ris:       single-layer kinds: 0 or 1 = area-uniform next points; 2..64 =
 *              resampled importance sampling from `ris` uniform candidates
 *              with target |kernel| (the paper uses 16).
 *   iter_limit: 0 = automatic (4 x wide BVH nodes + 64 node visits per
 *              line, which a line never needs: each node is visited at most
 *              once); a positive value bounds the visits per line lower.  A
 *              line that reaches the bound (or overflows the traversal stack)
 *              stops and sets the solve's check word: every estimate of that
 *              call is NaN and wob_solve_counted returns
 *              WOB_ERR_DEVICE_CHECK.  Small values exercise that path without
 *              any fault.
 */
typedef struct {
    wob_bvh bvh;
    int32_t kind;
    int32_t side;
    float alpha;
    int32_t data_mode;
    const float *vertex_data;
    float poly[10];
    float x0[3];
    float scale;
    uint32_t problem;
    float tau;
    const uint8_t *bc_type;
    float k_mix;
    float p_k;
    int32_t ris;
    int32_t iter_limit;
} wob_problem;

/* Per-walk and per-line outputs for parity checks (each pointer device, may
 * be NULL).  Line k of walk w of query q is entry (q * N + w) * M + k. */
typedef struct {
    double *per_walk;    /* Q x N walk values */
    uint8_t *walk_flag;  /* Q x N: 1 if any line of the walk was near-degenerate */
    int32_t *line_m;     /* Q x N x M hit counts, -1 for lines not traced */
    int32_t *line_prim;  /* Q x N x M picked triangle (original id), -1 for no hit
                            or a line not traced */
    uint8_t *line_flag;  /* Q x N x M: 1 if the line was near-degenerate */
} wob_debug_out;

/* Counters of the most recent wob_solve_counted() call. */
typedef struct {
    int64_t lines;        /* line queries (DL) or area samples (SL) issued */
    int64_t node_visits;  /* BVH interior nodes fetched */
    int64_t tri_tests;    /* triangles tested */
    int64_t hits;         /* intersections found */
    int64_t flagged;      /* near-degenerate lines */
} wob_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int wob_version(void);

/* Message for the calling thread's last error ("" if none). */
const char *wob_last_error(void);

/*
 * Upload a mesh and precompute per-triangle data (unit normals, areas and
 * the area prefix sums used by area sampling).  `verts`/`tris` are device
 * pointers if on_device != 0, host pointers otherwise; the library copies
 * them.  Validates the mesh (finite vertices, indices in [0, V), non-zero
 * areas, positive signed volume) and synchronises on `stream`.
 * Errors: WOB_ERR_INVALID_ARG, WOB_ERR_DEGENERATE_MESH, WOB_ERR_OOM, WOB_ERR_CUDA.
 */
int wob_build_mesh(const float *verts, int64_t V, const int32_t *tris, int64_t T,
                   int on_device, void *stream, wob_mesh *out);
int wob_mesh_get_info(wob_mesh m, wob_mesh_info *out);
void wob_destroy_mesh(wob_mesh m);

/*
 * Build the bounding-volume hierarchy used by the all-hits line queries of
 * ray sampling (Sec. 4.4.1): a linear BVH over Morton-ordered triangle
 * centroids (Karras 2012), bottom-up boxes, leaves of up to leaf_size
 * triangles, then collapsed top-down into 8-wide nodes (each node expands
 * its largest-area interior child until it has 8 children; child boxes
 * quantised to 8 bits, rounded outward).  Meshes whose binary tree has
 * 2^24 or more interior nodes are rejected (WOB_ERR_UNSUPPORTED).  The BVH
 * keeps a reference to the mesh; destroy the BVH first.  Synchronises on
 * `stream`.
 */
int wob_build_bvh(wob_mesh m, const wob_bvh_params *p, void *stream, wob_bvh *out);
int wob_bvh_get_info(wob_bvh b, wob_bvh_info *out);
void wob_destroy_bvh(wob_bvh b);

/*
 * Estimate u at Q query points with `walks` walks of at most `max_len`
 * boundary vertices each (Sec. 4.1.1, 4.1.2, 4.3):
 *   est[q] = mean of the walk values, var[q] = their unbiased sample variance
 *   (the standard error is sqrt(var / walks)).
 * queries: device, Q x 3 float.  query_prim: device, Q int32 (the triangle a
 * query lies on, -1 off the boundary) or NULL: for the single-layer kinds it
 * marks points on Gamma; for WOB_NEUMANN_DIRECT a query on triangle
 * query_prim[q] is the walk's first boundary vertex (weight 1) and the walk
 * estimates u there; for WOB_DIRICHLET_DL use wob_solve_density.
 * WOB_NEUMANN_DIRECT (Sec. 4.2): from a point off the boundary the first
 * line has weight phi (m/2) s and the source phi |Gamma| G(x0, x') q(x') at
 * an area-uniform x'; each boundary vertex has line weight phi m s and
 * source 2 phi |Gamma| G q, halved at the last vertex (Sec. 4.1.2); q is
 * dh/dn of the field (POLY, POINT) or the P1 vertex data.  Interior Neumann
 * solutions are defined up to a constant: the walks do not fix it.
 * est, var: device, Q doubles.  walks >= 2, 1 <= max_len <= 4096.
 * Allocates Q * ceil(walks / 32) * 16 bytes of scratch on `stream`
 * (stream-ordered): per query and block of 32 walks the sum and the sum of
 * squares of the walk values, added in a fixed order (results do not depend
 * on scheduling); var = (sum of squares - sum * mean) / (walks - 1).
 */
int wob_solve(const wob_problem *prob, const float *queries, const int32_t *query_prim,
              int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double *est,
              double *var, void *stream);

/*
 * Walks walk_begin .. walk_begin + walks - 1 only, ACCUMULATED into device
 * sum[q] += sum of walk values and sumsq[q] += sum of squares.  Calls over
 * disjoint walk ranges combine exactly into the result of one larger call
 * (up to summation order): the basis of progressive refinement.
 */
int wob_solve_range(const wob_problem *prob, const float *queries, const int32_t *query_prim,
                    int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len,
                    uint64_t seed, double *sum, double *sumsq, void *stream);

/*
 * Density of the double-layer representation at boundary points
 * (Eq. indirect_double_boundary_reordered2, Sec. 4.1.1): walks start ON the
 * boundary at points[q] (device, Q x 3) lying on triangle prims[q] (device,
 * original triangle ids); the point is vertex 1 (weight 1) and M - 1 lines
 * follow; est = mean of nu-hat, var = sample variance.  Only for
 * WOB_DIRICHLET_DL.  These are the training targets of the control variate.
 */
int wob_solve_density(const wob_problem *prob, const float *points, const int32_t *prims,
                      int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double *est,
                      double *var, void *stream);

/* As wob_solve, also writing the per-walk outputs of `dbg` (Q x walks);
 * for WOB_DIRICHLET_DL a non-NULL query_prim selects density walks as in
 * wob_solve_density. */
int wob_solve_debug(const wob_problem *prob, const float *queries, const int32_t *query_prim,
                    int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double *est,
                    double *var, const wob_debug_out *dbg, void *stream);

/*
 * Value and gradient of u at Q points off the boundary from the same walks
 * (Sec. 4.1.3, path reuse): only the first step's weight changes, from
 * -dG/dn_y / p = (m/2) s to -grad_x dG/dn_y / p = (m/2) s times
 * -(n - 3 (w . n) w) / (r (w . n)), with w = (x1 - x0) / r and n the normal
 * at the first hit (App. A).  The gradient weight grows as 1 / (w . n) at
 * grazing hits (a heavy-tailed estimator, as the paper observes near the
 * boundary).  WOB_DIRICHLET_DL only.  est, var: device, Q doubles;
 * grad_est, grad_var: device, 3 x Q doubles, component-major (component c of
 * query q at [c * Q + q]); per_walk_grad: optional device 3 x Q x walks
 * (component-major) per-walk gradients.  Allocates Q * walks * 4 doubles of
 * scratch on `stream`.
 */
int wob_solve_grad(const wob_problem *prob, const float *queries, int64_t Q, int32_t walks,
                   int32_t max_len, uint64_t seed, double *est, double *var, double *grad_est,
                   double *grad_var, double *per_walk_grad, void *stream);

/*
 * Forward (adjoint) estimator of single-layer Neumann problems (Sec. 4.4.3;
 * the boundary-sampling advantage of Sec. 5): `paths` paths start ON the
 * boundary at z_0 with weight 2 phi q(z_0) / p(z_0), follow lines as the
 * double-layer walks (all hits, one picked; weight phi m s per step) for
 * max_len vertices (the last weighted 1/2, Sec. 4.1.2), and every vertex is
 * connected to every query: u(x) = mean over paths of sum_j w_j G(x, z_j).
 * One set of paths serves all Q queries (cost ~ paths x max_len x Q for the
 * connections).  start_mode 0: z_0 area-uniform; 1: per triangle
 * proportional to area (|q(centroid)| + beta mean |q|), uniform on it -- the
 * boundary-value-weighted start for sparse data (beta > 0 keeps every
 * triangle reachable, so the estimate stays unbiased).  Expectation: that of
 * wob_solve for the same problem and max_len.  prob: WOB_NEUMANN_SL (phi
 * from side; ris is not used).  queries: device Q x 3; est, var: device Q
 * (var: unbiased variance of one path's contribution).  zpos (paths x
 * max_len x 3) and zw (paths x max_len), device, optional: the path
 * vertices and their weights (0 after a missed line); scratch for them is
 * allocated on `stream` when NULL.  path_flag (device, paths bytes,
 * optional): 1 if a line of the path was near-degenerate.  Paths draw from
 * the streams of query index = path index, walk index 0xFFFFFFFF.
 * 1 <= max_len <= 1024.
 */
int wob_solve_forward(const wob_problem *prob, const float *queries, int64_t Q, int32_t paths,
                      int32_t max_len, uint64_t seed, int32_t start_mode, float beta,
                      double *est, double *var, double *zpos, double *zw, uint8_t *path_flag,
                      void *stream);

/* As wob_solve, counting traversal work into *stats (synchronises).  The
 * counters are also kept for wob_get_stats. */
int wob_solve_counted(const wob_problem *prob, const float *queries, const int32_t *query_prim,
                      int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double *est,
                      double *var, wob_stats *stats, void *stream);

/* Counters (line queries, node visits, triangle tests, hits, near-degenerate
 * lines) of the most recent successful wob_solve_counted call of the calling
 * thread; all zero before the first.  Errors: WOB_ERR_INVALID_ARG (NULL). */
int wob_get_stats(wob_stats *out);

/*
 * wob_solve with HOST queries / query_prim / est / var: copies the inputs to
 * the device, solves, copies the results back and synchronises.  Device
 * buffers are allocated on `stream` and freed before returning.
 */
int wob_solve_host(const wob_problem *prob, const float *queries_host,
                   const int32_t *query_prim_host, int64_t Q, int32_t walks, int32_t max_len,
                   uint64_t seed, double *est_host, double *var_host, void *stream);

/*
 * Batched solves: P independent double-layer Dirichlet problems (each with
 * its own mesh/BVH, data, walks and path length) run as ONE persistent
 * launch, captured in a CUDA graph at creation and replayed by
 * wob_batch_run.  The walks are cut into tiles of 32 * tile_rounds walks of
 * one problem; warps take tiles from a global counter (one atomic per
 * tile), so a warp always works on a single problem (one BVH, one path
 * length).  Results equal P separate wob_solve calls with the same seed and
 * the problems' own `problem` indices.
 *   problems:      host array of P descriptors (kind must be WOB_DIRICHLET_DL)
 *   query_offsets: host, P + 1; problem p owns queries/est/var rows
 *                  [query_offsets[p], query_offsets[p+1])
 *   walks, max_len: host, P each (walks >= 2, 1 <= max_len <= 4096)
 *   queries:       device, query_offsets[P] x 3 float; est, var: device,
 *                  query_offsets[P] doubles -- bound to the batch
 *   params:        schedule; NULL or autotune = 1 times the candidate
 *                  schedules once on this batch (walk counts scaled down)
 *                  and caches the choice in $WOB_TUNE_CACHE (default
 *                  ~/.cache/wob_autotune.json), keyed by GPU and batch shape
 * The batch allocates Q_total * ceil(walks / 32) * 16 bytes of scratch (sum
 * and sum of squares per query and block of 32 walks) at creation and keeps
 * it until wob_batch_destroy.  The BVHs must outlive the batch.
 */
typedef struct wob_batch_s *wob_batch;

typedef struct {
    int32_t tile_rounds; /* tile = 32 * tile_rounds walks (1, 2 or 4) */
    int32_t order;       /* 0: problem after problem; 1: costliest problems first */
    int32_t autotune;    /* 1: choose tile_rounds and order by timing */
    int32_t reserved[5];
} wob_batch_params;

typedef struct {
    int32_t P;
    int32_t tile_rounds;
    int32_t order;
    int32_t from_cache;    /* schedule read from the autotune cache */
    int64_t queries;       /* total queries */
    int64_t walks;         /* total walks */
    int64_t max_lines;     /* total walks x their path lengths (upper bound) */
    int64_t tiles;
    double tune_ms[8];     /* measured candidates (tile_rounds x order), 0 if not run */
} wob_batch_info;

/*
 * One-shot batched solve: P double-layer problems (Sec. 4.1) in one
 * persistent launch, with the arguments of wob_batch_create and the seed of
 * wob_batch_run (schedule from the autotune cache, timed on first use).
 * Equivalent to wob_batch_create + wob_batch_run + wob_batch_destroy;
 * synchronises on `stream`.  est / var receive, per problem p, rows
 * query_offsets[p] .. query_offsets[p+1] - 1.  Results equal P separate
 * wob_solve calls with the same seed and the problems' own `problem` indices.
 */
int wob_solve_batched(const wob_problem *problems, int32_t P, const int64_t *query_offsets,
                      const float *queries, const int32_t *walks, const int32_t *max_len,
                      uint64_t seed, double *est, double *var, void *stream);

int wob_batch_create(const wob_problem *problems, int32_t P, const int64_t *query_offsets,
                     const int32_t *walks, const int32_t *max_len, const float *queries,
                     double *est, double *var, const wob_batch_params *params, void *stream,
                     wob_batch *out);
/* Replay the batch's graph on `stream` with this seed. */
int wob_batch_run(wob_batch b, uint64_t seed, void *stream);
int wob_batch_get_info(wob_batch b, wob_batch_info *out);
void wob_batch_destroy(wob_batch b);

/*
 * Learned control variate (not in the paper; it reuses the double-layer
 * representation of Sec. 3.3 and Table 1).  With nu = nu_t + rho, where
 * nu_t is a network, rho solves rho = H rho + r with
 *     r = 2 phi g - nu_t + H nu_t,   and   u(x0) = D nu_t(x0) + D rho(x0),
 * (H f)(x) = 2 phi int dG/dn_y f dA, (D f)(x0) = -int dG/dn_y f dA.  The
 * walks estimate only D rho; D nu_t and H nu_t are computed by quadrature
 * (Radon's 7-point degree-5 rule per triangle; triangles whose centroid is
 * within `near` x their longest edge of the target use 4^level
 * sub-triangles; H subtracts nu_t(x) and adds H[1] = -phi).  Any nu_t keeps
 * the estimator unbiased up to quadrature error; a good one makes r small.
 *
 * Network: 96 Fourier features (sin, cos of 2 pi 2^(k/3) y_d, k = 0..15,
 * column 32 d + 2 k + {0: sin, 1: cos}) -> 4 x (64, SiLU) -> 1; parameters
 * FP32 (device), layer by layer: W (out x in, row-major) then b; BF16
 * tensor-core arithmetic with FP32 accumulation.
 */
int wob_mlp_num_params(void); /* 18753 */
/* He-uniform initial parameters (device, n_params floats): weight i (flat
 * index) of a layer with fan-in f is sqrt(6 / f) (2 u - 1), u = (x >> 8) 2^-24
 * for x the first word of the Philox4x32-10 block with counter (i, 0,
 * 3 << 12, 0) and key (seed, seed >> 32); biases 0. */
int wob_mlp_init(float *params, uint64_t seed, void *stream);
/* out[i] = network(x[i]), x device n x 3, out device n. */
int wob_mlp_forward(const float *params, const float *x, int64_t n, float *out, void *stream);
/* One step on the mean squared error of (network(x), target) over the n
 * samples: gradients (deterministic, block order), then Adam (b1 0.9, b2
 * 0.999, eps 1e-8, bias-corrected, `step` >= 1) on params / adam_m /
 * adam_v unless lr == 0.  grad_out (n_params floats) and loss_out (1 float)
 * are optional device outputs. */
int wob_mlp_train_step(float *params, float *adam_m, float *adam_v, const float *x,
                       const float *target, int64_t n, float lr, int32_t step, float *grad_out,
                       float *loss_out, void *stream);

/* Test hook: the tensor-core network kernels give up the first wait on
 * each product after `polls` mbarrier polls (default 2^26, about a second);
 * a kernel that gives up waits (bounded) for its products in flight, frees
 * its tensor memory and writes NaN outputs (forward) or NaN gradients and
 * loss (training), and the context stays usable.  0 makes every first wait
 * give up at once.  Process-wide; the previous value is returned in
 * *previous (optional).  Calls in flight keep the value they started with. */
int wob_debug_set_tc_wait_limit(uint32_t polls, uint32_t *previous);

typedef struct wob_cv_s *wob_cv;
/* Quadrature nodes for a mesh (level 0..3, near > 0); node values start at 0.
 * Synchronises.  The mesh must outlive the object. */
int wob_cv_create(wob_mesh m, int32_t level, float near, void *stream, wob_cv *out);
/* Node values = the network at every node. */
int wob_cv_set_network(wob_cv c, const float *params, void *stream);
/* Node values given directly (device; T x 7 coarse, T x F fine). */
int wob_cv_set_node_values(wob_cv c, const float *coarse, const float *fine, void *stream);
/* Copy the nodes (x, y, z, weight per node; T x 7 coarse, T x F fine) into
 * caller device buffers of 4 floats per node. */
int wob_cv_get_nodes(wob_cv c, float *coarse_out, float *fine_out, void *stream);
int wob_cv_get_info(wob_cv c, int32_t *T, int32_t *F, int64_t *candidates);
/* D f at n points off the surface / H f at n points on triangles prims with
 * f(x) = fx (all device). */
int wob_cv_quad_D(wob_cv c, const float *points, int64_t n, float *out, void *stream);
int wob_cv_quad_H(wob_cv c, int32_t phi, const float *points, const int32_t *prims,
                  const float *fx, int64_t n, float *out, void *stream);
/* Residual walks walk_begin .. walk_begin + walks - 1 of Q queries:
 * sum[q] += sum of walk values, sumsq[q] += sum of squares (as
 * wob_solve_range); per_walk (Q x walks, optional) receives the values and
 * dnt (Q floats, optional) D nu_t at the queries.  The estimate is
 * dnt[q] + sum[q] / total walks.  prob: WOB_DIRICHLET_DL on c's mesh; the
 * node values must come from the same `params` (wob_cv_set_network). */
int wob_cv_solve(const wob_problem *prob, wob_cv c, const float *params, const float *queries,
                 int64_t Q, int64_t walk_begin, int32_t walks, int32_t max_len, uint64_t seed,
                 double *sum, double *sumsq, double *per_walk, float *dnt, void *stream);
void wob_cv_destroy(wob_cv c);

/*
 * Residual walks with Monte Carlo integrals, for meshes too large for the
 * quadrature of wob_cv_solve (no wob_cv object: nothing scales with the
 * mesh size but the traversal).  With nu = nu_t + rho (Table 1, Dirichlet
 * double layer) the walk value is
 *     D^ nu_t (x0) + sum_k P_k c_k [2 phi g(x_k) - nu_t(x_k) + H^ nu_t (x_k)],
 * the walk's own recursion (Sec. 4.1, the 1/2 on the last vertex of
 * Sec. 4.1.2) with the residual source, where D^ and H^ are means of K
 * one-line estimates: K independent all-hits lines from the point (Sec.
 * 4.4.1), each picking y_j with the walk's own line weight -- (m/2) s from
 * the query, -phi m s from a boundary vertex -- times nu_t(y_j).  Unbiased
 * for the truncated residual series; nu_t = 0 gives plain WoB.  Extra line
 * j of vertex v (0 = the query) of walk w draws from the streams
 * (query, w | 2^31, v K + j).  params: the network (device, wob_mlp_num_params
 * floats).  sum / sumsq: device Q doubles, accumulated (+=) as in
 * wob_solve_range; per_walk (device Q x walks, optional).  1 <= K <= 16,
 * max_len <= 1024, walk indices below 2^31, Q x walks x K < 2^31 per call.
 * Scratch: about Q x walks x (76 + 20 K) bytes, allocated on `stream`.
 */
int wob_cv_solve_mc(const wob_problem *prob, const float *params, const float *queries, int64_t Q,
                    int64_t walk_begin, int32_t walks, int32_t max_len, int32_t K, uint64_t seed,
                    double *sum, double *sumsq, double *per_walk, void *stream);

/*
 * Area-uniform points on the mesh (device outputs: points n x 3 float,
 * prims n original triangle ids).  Point i is the area sample of the
 * counter-based stream (query i, walk 0, step 0) under key (seed ^ problem,
 * seed >> 32): triangle by inverse CDF of the areas, then the square-root
 * warp b = (1 - sqrt(u1), sqrt(u1)(1 - u2), sqrt(u1) u2) -- the draw the
 * single-layer walks make (Sec. 4.3 with uniform area sampling).  0 <= n < 2^31.
 */
int wob_sample_boundary(wob_mesh m, int64_t n, uint64_t seed, uint32_t problem, float *points,
                        int32_t *prims, void *stream);

/*
 * Train the control variate's network nu_t on density estimates, then set
 * c's node values from it.  Training set: `points` area-uniform boundary
 * points (wob_sample_boundary with point_seed and prob->problem); target at
 * each = mean of `walks` density walks of length max_len (wob_solve_density
 * with walk_seed).  Then `epochs` passes of Adam (lr) over minibatches of
 * `batch` consecutive points (the points are independent draws, so fixed
 * order is a valid stochastic gradient) at rate lr, the last tail_epochs of
 * them at lr_end; the Adam step counter starts at step0 + 1.  params /
 * adam_m / adam_v (device, n_params floats each) are updated in place;
 * loss_out (device, optional) receives the minibatch MSE of every step,
 * epochs x ceil(points / batch) floats.  One epoch of steps is captured as
 * a CUDA graph (on a stream of the library's own) and replayed on `stream`
 * once per epoch; the call synchronises `stream` before returning.  The
 * library allocates about points x 36 bytes of scratch on `stream` and
 * frees it before returning.  prob: WOB_DIRICHLET_DL on c's mesh.
 */
typedef struct {
    int64_t points;      /* training points (1 .. 2^31 - 1) */
    int32_t walks;       /* density walks per point (>= 2) */
    int32_t max_len;     /* their path length M */
    uint64_t point_seed; /* seed of the training points */
    uint64_t walk_seed;  /* seed of the density walks */
    int32_t epochs;      /* >= 0 */
    int32_t batch;       /* minibatch size, 1 .. 2^22 */
    float lr;            /* Adam learning rate, >= 0 */
    float lr_end;        /* rate of the last tail_epochs epochs, >= 0 */
    int32_t tail_epochs; /* 0: lr throughout */
    int32_t step0;       /* Adam steps already taken with adam_m / adam_v */
} wob_cv_train_params;

int wob_cv_train(const wob_problem *prob, wob_cv c, const wob_cv_train_params *tp,
                 float *params, float *adam_m, float *adam_v, float *loss_out, void *stream);

/*
 * wob_solve for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of wob_solve.  wob_solve
 * allocates one double per walk of scratch on every call; a caller whose
 * process has handed the GPU's memory to its own allocator, or that cannot
 * afford an allocation and the synchronisation it may imply on its path,
 * calls this instead.  The per-walk values live in a fixed array inside the
 * library (2^20 doubles = 8 MiB, held on every GPU that loads the library's
 * device code until exit), so:
 *   - Q * ceil(walks / 32) must be <= 2^19 (the array holds a sum and a sum
 *     of squares per query and block of 32 walks; else WOB_ERR_INVALID_ARG,
 *     nothing launched);
 *   - no cudaMalloc, cudaFree or other allocating routine is called;
 *   - all calls share that array: calls that overlap on the GPU (other
 *     streams or host threads) race; serialise them;
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after a cudaDeviceReset (or any other end of the device's
 *     primary context) it is stale, so do not call this entry point again.
 * Arguments, outputs and results are those of wob_solve (bit-identical).
 */
int wob_solve_noalloc(const wob_problem *prob, const float *queries, const int32_t *query_prim,
                      int64_t Q, int32_t walks, int32_t max_len, uint64_t seed, double *est,
                      double *var, void *stream);

/*
 * All-hits queries of n explicit lines {o + t d, t real} (Sec. 4.4.1), all
 * pointers device.  origins/dirs: n x 3 double (dirs unit length).
 * exclude: n int32 triangle ids skipped (the point's own face), or NULL.
 * keys: n x 3 uint32 (query, walk, step) addressing the hit-selection keys.
 * Outputs (n each, any may be NULL except m): hit count m, sum of
 * s = sign(omega . n) over all hits, picked triangle id (-1 if none), its s,
 * its line parameter t and point y (n x 3), and the near-degenerate flag.
 */
int wob_trace_lines(wob_bvh b, const double *origins, const double *dirs,
                    const int32_t *exclude, const uint32_t *keys, int64_t n, uint64_t seed,
                    uint32_t problem, float tau, int32_t *m, int32_t *sum_s, int32_t *prim,
                    int32_t *s, double *t, double *y, uint8_t *flag, void *stream);

/* Line axes of the walks' streams, for (query, walk, step) triples (device,
 * n x 3) -> device n x 3 doubles.  Marsaglia (1972) sampling of the unit
 * sphere, formed in FP64 (the walk kernels carry the same axis as a
 * float-float pair, equal to it within about 2^-44 relative). */
int wob_line_axes(uint64_t seed, uint32_t problem, const uint32_t *qws, int64_t n, double *d,
                  void *stream);

/* Raw Philox4x32-10 blocks: ctr n x 4, key n x 2, out n x 4 (device). */
int wob_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out,
                      void *stream);

/*
 * Measurement probe (the paper has no counterpart): `passes` streaming reads
 * of the device buffer buf (bytes, a multiple of 16, 16-byte aligned) with
 * 16-byte loads that bypass L1, by a grid of resident blocks on every SM;
 * the sum of the read floats goes to *out (device float, overwritten).  Timed
 * around the call on a buffer that fits in L2, it gives the L2 read
 * bandwidth the line traversal's node fetches are measured against.
 * Errors: WOB_ERR_INVALID_ARG (bad size or alignment), WOB_ERR_CUDA.
 */
int wob_probe_l2_read(const void *buf, int64_t bytes, int32_t passes, float *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* WOB_H */
