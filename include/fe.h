/*
 * fe.h -- C ABI of a GB300 (sm_103a) library for finite-element numerical
 * integration with first-order elements: per-element stiffness matrices A^e and
 * load vectors b^e for linear tetrahedra and linear 6-node prisms.
 *
 * The operation is the one of Banas, Kruzel, Bielanski, arXiv 1504.01023:
 *   (A^e)^{rs} = int_{Omega_e} ( c^{i;j} phi^r_{,i} phi^s_{,j} + c^{i;0} phi^r_{,i} phi^s
 *                               + c^{0;i} phi^r phi^s_{,i} + c^{0;0} phi^r phi^s ) dOmega
 *   (b^e)^{r}  = int_{Omega_e} ( d^i phi^r_{,i} + d^0 phi^r ) dOmega
 * (Sec. 2.2, Eqs. sm_local and lv_local), evaluated through the reference element
 * (Eq. change_of_variables) with Gaussian quadrature (Eq. quadrature), following
 * the generic procedure of Algorithm 1 and its QSS orderings (Algorithms 2, 3).
 * Boundary terms are not computed (Sec. 2.1 neglects them).
 *
 * Conventions used by every entry point
 *  - No exception crosses the ABI; every call returns an fe_status.
 *  - Pointers marked "device" are CUDA device pointers of the context's device,
 *    owned by the caller unless stated otherwise. Pointers marked "host" are plain
 *    host memory (pinned memory makes the copies asynchronous).
 *  - A `stream` argument is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Work is enqueued on it; the call returns after the enqueue.
 *    Asynchronous device errors are reported by fe_ctx_sync, fe_serve_poll or the
 *    next call on the context.
 *  - Index 0 of the coefficient arrays means the function value, 1..3 the x,y,z
 *    derivatives: C[a][b] (a,b = 0..3) holds c^{a;b}, D[a] holds d^a. Row r of A^e
 *    is the test function, column s the trial function.
 *  - Reference elements and node order: tetrahedron {xi,eta,zeta >= 0,
 *    xi+eta+zeta <= 1} with shape functions 1-xi-eta-zeta, xi, eta, zeta for
 *    vertices 0..3; prism = triangle {xi,eta >= 0, xi+eta <= 1} x zeta in [-1,1],
 *    vertices 0..2 the bottom triangle (zeta = -1) and 3..5 the top one, vertex
 *    k+3 above vertex k.
 *  - A context is used by one host thread at a time, except fe_serve_submit,
 *    fe_serve_poll, fe_serve_wait_any and fe_serve_release, which may be called
 *    from any thread.
 */
#ifndef FE_H_
#define FE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FE_ABI_VERSION 1

typedef enum fe_status {
    FE_OK = 0,
    FE_NOT_READY = 1,          /* serving: the request has not finished yet */
    FE_ERR_INVALID_ARG = -1,   /* a pointer, size, enum or layout is not valid */
    FE_ERR_OOM = -2,           /* a device or host allocation failed */
    FE_ERR_BUDGET = -3,        /* serving: the request can never fit the HBM budget */
    FE_ERR_CUDA = -4,          /* a CUDA runtime call failed (text in fe_last_error) */
    FE_ERR_TIMEOUT = -5,       /* a bounded device wait ran out */
    FE_ERR_UNSUPPORTED = -6,   /* valid but not implemented combination */
    FE_ERR_PARTIAL = -7        /* tiles were skipped (injected fault only): outputs incomplete */
} fe_status;

typedef enum fe_elem_type { FE_TET = 0, FE_PRISM = 1 } fe_elem_type;

/* Sec. 4.1: "Poisson" = Laplace operator (c^{i;j} = delta_ij, no other c),
   d^0 per integration point; "conv-diff" (here FE_GENERIC) = all 16 c and 4 d. */
typedef enum fe_problem { FE_POISSON = 0, FE_GENERIC = 1 } fe_problem;

/* FE_FP64: all arithmetic in double, inputs and outputs double.
   FE_FP32_MIXED: coordinates stay double in memory; edge vectors are formed
   exactly enough in single precision, the coefficient and shape-derivative
   arithmetic and accumulation run in float, coefficients and outputs are float.
   Elements that fail a mean-ratio shape test (quality < 0.1) get their Jacobian,
   determinant and inverse in double (flag bit 0).
   FE_FP64_DW: double inputs and outputs and double accuracy (the FE_FP64
   tolerance), computed in double-word arithmetic (pairs of floats, about 48
   significant bits) on the float pipes, with the edge vectors x_k - x_0 formed in
   double. Elements that fail the shape test above, or whose |det J|, inputs or
   results leave the double-word window (|det J| in [2^-60, 2^60], nonzero
   coefficients in [2^-50, 2^51), the sum of |A^e| and of |b^e| zero or in
   [2^-80, 2^100]), are computed entirely in double (flag bit 0). The paper has
   no counterpart: its double-precision form is FE_FP64. */
typedef enum fe_precision { FE_FP64 = 0, FE_FP32_MIXED = 1, FE_FP64_DW = 2 } fe_precision;

/* Gaussian rules (Sec. 2.3; the paper names no points, these are the readings):
   TET1   centroid, weight 1/6 (degree 1);
   TET4   barycentric permutations of (b,a,a,a), a=(5-sqrt5)/20, b=(5+3sqrt5)/20,
          weights 1/24 (degree 2);
   PRISM6 triangle {(1/6,1/6),(2/3,1/6),(1/6,2/3)} weights 1/6 x Gauss-Legendre
          zeta = -+1/sqrt3 weights 1. */
typedef enum fe_quad { FE_QUAD_TET1 = 0, FE_QUAD_TET4 = 1, FE_QUAD_PRISM6 = 2 } fe_quad;

/* Sec. 3.3 takes coefficients constant per element; per integration point is the
   input mode of the prism workload with varying coefficients. */
/* FE_COEF_FUNCTION_U: the coefficients at each integration point come from a
   problem-dependent function (Sec. 2.3 input list; Sec. 3.1) of a field u given by
   its nodal values: coefs holds u_k, NS per element (element-contiguous, in the
   coefficient precision), u_Q = sum_k phi_k(xi_Q) u_k, and coefficient j (0..15
   C[4][4] row-major, 16..19 D[4]) at Q is P[0][j] + P[1][j] u_Q + P[2][j] u_Q^2
   with P = *coef_fn. The Laplace kind uses slot 16 (d^0) only. For nonlinear
   problems (c(u)) re-integrated at each iterate without materialising the
   coefficients. */
typedef enum fe_coef_mode { FE_COEF_PER_ELEMENT = 0, FE_COEF_PER_QPOINT = 1, FE_COEF_FUNCTION_U = 2 } fe_coef_mode;

typedef struct fe_coef_function {
    double p[3][20];
} fe_coef_function;

/* Sec. 4.2 (Figs. 1, 2): SOA = one plane per scalar, elements contiguous inside a
   plane ("coalesced" order); AOS = the "natural" order, all scalars of one
   element contiguous. */
/* FE_LAYOUT_INDEXED (coordinates only): a shared node array plus an element ->
   node table, the global structures the integration loop reads its geometry
   from (Sec. 3.1); see fe_elem_args. */
typedef enum fe_layout { FE_LAYOUT_SOA = 0, FE_LAYOUT_AOS = 1, FE_LAYOUT_INDEXED = 2 } fe_layout;

typedef enum fe_memory { FE_MEM_DEVICE = 0, FE_MEM_HOST = 1 } fe_memory;

typedef struct fe_ctx fe_ctx;

typedef struct fe_ctx_config {
    int device;                    /* CUDA device ordinal */
    uint64_t hbm_budget_bytes;     /* serving admission budget; 0 = 120e9 bytes */
    int serve_slots;               /* serving launches in flight at once; 0 = 4, at most 64 */
    int autotune;                  /* 1: time the candidate launch shapes of a key on
                                      its first use and keep the fastest */
    const char *tuning_cache_path; /* text file holding tuned shapes; NULL = none */
} fe_ctx_config;

/*
 * Inputs of one element set of a single type (Sec. 2.3, input list): geometry
 * degrees of freedom (vertex coordinates), the coefficients, the rule.
 *
 * coords (double, always): NS = 4 (tet) or 6 (prism) vertices x 3 coordinates.
 *   SOA: scalar j = 3*v + d lives at coords[j*coords_stride + e].
 *   AOS: coords[(e*NS + v)*3 + d].
 *   INDEXED: coords is the node array, node i at coords[3*i + d], i < n_nodes,
 *     and vertex v of element e is node conn[e*NS + v] (int32, 0-based). Device
 *     memory only; coefficients element-contiguous (coefs_layout AOS); the
 *     batched and serving entry points do not take it. An index outside
 *     [0, n_nodes) is not read: that element's A^e and b^e are zero and its
 *     flag has bit 3 set.
 * coefs (double for FE_FP64 and FE_FP64_DW, float for FE_FP32_MIXED), NC scalars per element:
 *   FE_GENERIC: 20 per point (C[4][4] row-major, then D[4]); FE_POISSON: 1 per
 *   point (d^0). NC = that count times NQ for FE_COEF_PER_QPOINT (point-major:
 *   scalar j = q*per_point + k), times 1 for FE_COEF_PER_ELEMENT.
 *   SOA: scalar j at coefs[j*coefs_stride + e]; AOS: coefs[e*NC + j].
 * A stride of 0 means n_elem. SOA strides are counted in elements, at most 2^40.
 */
typedef struct fe_elem_args {
    int64_t n_elem;
    const double *coords;
    fe_layout coords_layout;
    int64_t coords_stride;
    fe_problem kind;
    fe_quad quad;
    fe_coef_mode coef_mode;
    const void *coefs;
    fe_layout coefs_layout;
    int64_t coefs_stride;
    fe_precision prec;
    fe_memory memory;              /* where coords and coefs live */
    const int32_t *conn;           /* FE_LAYOUT_INDEXED: [n_elem][NS] node indices, device */
    int64_t n_nodes;               /* FE_LAYOUT_INDEXED: nodes in coords, < 2^31 */
    int ordering;                  /* loop ordering (Sec. 3.3): 0 QSS (Algorithms 2, 3; the default),
                                      1 SQS (Algorithms 4, 5), 2 SSQ (Algorithms 6, 7). SQS and SSQ are
                                      for comparison: FE_FP32_MIXED, element-contiguous (AOS)
                                      coordinates and full AOS outputs only */
    const fe_coef_function *coef_fn; /* FE_COEF_FUNCTION_U: host, read during the call;
                                        element-contiguous (AOS) coordinates, full outputs,
                                        ordering 0; not for batches, serving, noalloc */
} fe_elem_args;

/*
 * Outputs (Sec. 4.2, Fig. 2): A^e full NS x NS, row-major entry k = r*NS + s
 * (NA = NS*NS entries), or, with packed = 1 (FE_POISSON only, whose A^e is
 * symmetric), its upper triangle row by row: entry k = r*NS - r*(r-1)/2 + (s - r)
 * for s >= r (NA = NS*(NS+1)/2: 10 for tetrahedra, 21 for prisms); b^e NS
 * entries. Element type: double (FE_FP64, FE_FP64_DW) or float.
 *   SOA ("coalesced"): A[k*stride + e], b[r*stride + e].
 *   AOS (element-contiguous): A[e*NA + k], b[e*NS + r].
 * packed = 1 is not accepted with FE_LAYOUT_INDEXED coordinates, by the batched
 * and serving entry points or by fe_integrate_tet_noalloc (FE_ERR_UNSUPPORTED).
 * flags (optional, may be NULL): one byte per element, bit 0 = the double
 * Jacobian path was used, bit 1 = det J < 0 somewhere (|det J| is integrated),
 * bit 2 = degenerate (|det J| <= 1e-300 in double): A^e = 0 and b^e = 0,
 * bit 3 = a node index outside the node array (FE_LAYOUT_INDEXED): A^e = 0, b^e = 0.
 */
typedef struct fe_out {
    void *A;
    void *b;
    fe_layout layout;
    int64_t stride;
    uint8_t *flags;
    fe_memory memory;              /* where A, b and flags live */
    int packed;                    /* 1: upper triangle of a symmetric A^e (FE_POISSON) */
} fe_out;

/* Create a context on cfg->device (NULL cfg = device 0, defaults). Allocates the
   context's scratch (fix-up lists, status words) and streams. */
fe_status fe_ctx_create(const fe_ctx_config *cfg, fe_ctx **out);
/* Stop serving, free every resident mesh, output and scratch buffer. */
fe_status fe_ctx_destroy(fe_ctx *ctx);
/* Wait for all work of the context and report the first asynchronous error. */
fe_status fe_ctx_sync(fe_ctx *ctx);
/* Text of the last error on this context (thread-local when ctx is NULL). */
const char *fe_last_error(fe_ctx *ctx);

/*
 * Integrate n_elem tetrahedra (Algorithm 3, QSS_geo_linear: the Jacobian terms
 * are formed once per element) / n_elem prisms (Algorithm 2, QSS_geo_generic:
 * the Jacobian terms are formed at each integration point).
 * Quadrature: tet FE_QUAD_TET1 or FE_QUAD_TET4; prism FE_QUAD_PRISM6.
 * With memory = FE_MEM_HOST (inputs and/or outputs) the call returns once the
 * outputs are in host memory. If every host buffer is pinned (page-locked and
 * mapped), the kernels read and write it in place over the host link (no
 * copies); otherwise the call copies through device staging buffers of the
 * context in chunks, overlapping the copies with the kernels.
 * Errors: FE_ERR_INVALID_ARG (null or misaligned pointer, stride < n_elem, quad
 * not valid for the type), FE_ERR_OOM (staging or scratch growth failed),
 * FE_ERR_CUDA. n_elem = 0 is valid and does nothing.
 */
fe_status fe_integrate_tet(fe_ctx *ctx, const fe_elem_args *args, const fe_out *out, void *stream);
fe_status fe_integrate_prism(fe_ctx *ctx, const fe_elem_args *args, const fe_out *out, void *stream);

/*
 * Matrix-free application (the element matrices consumed where they are
 * computed, never stored; the paper leaves their use to the solver, Sec. 2.2):
 *   y[conn[e][r]] += sum_s A^e_rs x[conn[e][s]]   and, if f != NULL,
 *   f[conn[e][r]] += b^e_r,                        for every element e and r.
 * args must use FE_LAYOUT_INDEXED geometry (device memory). x, y and f are device
 * arrays of n_nodes values, double for FE_FP64 and FE_FP64_DW, float for
 * FE_FP32_MIXED; y and f accumulate (zero them first for a plain product), by
 * atomic additions, so the order of the sums, and the last bits of the result,
 * vary between calls. flags (optional, device, n_elem bytes) as for
 * fe_integrate_*. An element whose node index is out of range adds nothing
 * (flag bit 3); flagged elements of the mixed and double-word forms add their
 * double-precision results once. Enqueued on `stream`.
 */
fe_status fe_apply_tet(fe_ctx *ctx, const fe_elem_args *args, const void *x, void *y, void *f, uint8_t *flags,
                       void *stream);
fe_status fe_apply_prism(fe_ctx *ctx, const fe_elem_args *args, const void *x, void *y, void *f, uint8_t *flags,
                         void *stream);

/* Host-only argument validation used by the calls above (no CUDA call). */
fe_status fe_check_args(fe_elem_type type, const fe_elem_args *args, const fe_out *out);

/* The quadrature the kernels use (Sec. 2, Eq. quadrature): for each of the rule's
   points its weight (weights[q], reference-element measure) and the reference
   shape-function values there (shape_values[q * NS + r], NS = 4 or 6, vertex r
   of the element record). Host arrays of max_points (x NS) entries; NULL skips
   an array. Host-only; needs no device. */
fe_status fe_rule_table(fe_quad quad, int max_points, int *n_points, double *weights, double *shape_values);

/* Algorithmic bytes moved per element (inputs read once, outputs written once):
   8*3*NS for coordinates + coefficient bytes + (NS*NS + NS) output scalars; the
   double-precision cases of Table 3 give 288, 528, 416, 640. -1 if invalid. */
int64_t fe_bytes_per_element(fe_elem_type type, fe_problem kind, fe_quad quad, fe_coef_mode mode,
                             fe_precision prec);

/*
 * Resident meshes (Sec. 3.1: element data kept in the memory of the processor
 * doing the integration). Copies geometry (host or device source, SOA planes of
 * stride n_elem or AOS records) into a context-owned element-contiguous (AOS)
 * device buffer and returns its id. Counted against the HBM budget
 * (FE_ERR_BUDGET if it does not fit). Releasing waits for the device.
 */
fe_status fe_mesh_register(fe_ctx *ctx, fe_elem_type type, int64_t n_elem, const double *coords,
                           fe_layout layout, fe_memory memory, int64_t *mesh_id);
fe_status fe_mesh_release(fe_ctx *ctx, int64_t mesh_id);

/*
 * Batched integration: many element sets of uneven size and mixed type, kind,
 * rule and coefficient mode in one step (not in the paper, which runs one
 * homogeneous set per kernel, Sec. 3.2): one persistent kernel per combination
 * (type, kind, rule, coefficient mode) present, all on parallel branches of one
 * CUDA graph, so that each combination's blocks fill the SMs the others leave
 * idle. Blocks take tiles of consecutive elements from their combination's
 * counter; tiles are ordered by decreasing size. The launch sequence {counter
 * reset, the combinations' persistent kernels, fix-up kernel} is captured into
 * the graph on the first submission of an item list (same items
 * byte for byte, i.e. same pointers and sizes) and replayed on later ones; the
 * last 8 lists are kept. With autotune on, the first submission times each
 * combination present on its own with tiles of 64, 128 and 256 elements,
 * persistent grids (blocks take tiles from the combination's counter) or one
 * block per tile, and for prisms one or two threads per element (as described at
 * fe_tune), and keeps the fastest shape of each combination; without, 128
 * elements, persistent, one thread. fe_batch_set_shape pins one shape for all
 * combinations instead.
 * Items must be FE_FP32_MIXED, device memory, element-contiguous (AOS) inputs
 * and outputs (FE_ERR_UNSUPPORTED otherwise). At most 2^23 items.
 */
typedef struct fe_batch_item {
    fe_elem_type type;
    fe_elem_args args;
    fe_out out;
} fe_batch_item;
fe_status fe_batch_submit(fe_ctx *ctx, const fe_batch_item *items, int n_items, void *stream);

/*
 * Serving (no counterpart in the paper, whose kernels run one element set per
 * call, Sec. 3.2): integration requests on resident meshes arrive at any time. A
 * scheduler thread admits them in arrival order while the resident meshes plus
 * the outputs of admitted, unreleased requests fit the HBM budget, merges every
 * admitted mixed-precision request into one batched launch (continuous
 * batching), runs FE_FP64 and FE_FP64_DW requests as their own launches, and keeps up to
 * serve_slots launches in flight on separate streams, so requests that arrive
 * while others run overlap with them on the device. coefs is a device pointer,
 * element-contiguous (AOS), float for FE_FP32_MIXED and double otherwise. The
 * outputs are context-owned element-contiguous device buffers, valid until
 * fe_serve_release.
 */
typedef struct fe_request {
    int64_t mesh_id;
    fe_problem kind;
    fe_quad quad;
    fe_coef_mode coef_mode;
    const void *coefs;
    fe_precision prec;
} fe_request;

typedef struct fe_result {
    fe_status status;
    fe_elem_type type;
    int64_t n_elem;
    void *A;                       /* device, AOS [n_elem][NS][NS], context-owned */
    void *b;                       /* device, AOS [n_elem][NS] */
    uint8_t *flags;                /* device, [n_elem] */
    double t_submit_us;            /* host steady clock, microseconds */
    double t_launch_us;            /* when the scheduler enqueued its launch */
    double t_done_us;              /* stamped by a host callback when its stream finished */
} fe_result;

/* Queue a request; FE_ERR_BUDGET if its outputs could never fit. Thread-safe. */
fe_status fe_serve_submit(fe_ctx *ctx, const fe_request *req, uint64_t *ticket);
/* FE_NOT_READY while waiting or running; FE_OK with res filled when done.
   Thread-safe. */
fe_status fe_serve_poll(fe_ctx *ctx, uint64_t ticket, fe_result *res);
/* Withdraw a request that has not been launched yet: FE_OK and its ticket is
   forgotten. FE_ERR_INVALID_ARG if the ticket is unknown or the request is
   already running or done (release it once it is done). Thread-safe. */
fe_status fe_serve_cancel(fe_ctx *ctx, uint64_t ticket);
/* Free a finished request's outputs and return their bytes to the budget. */
fe_status fe_serve_release(fe_ctx *ctx, uint64_t ticket);
/* Several requests at once (host arrays of n entries), under one lock and one
   scheduler wake-up, so that requests submitted together can share one launch.
   All or nothing: if any request is invalid (as fe_serve_submit would reject it),
   none is queued and the status is that request's; tickets[] is written only on
   FE_OK. n = 0 does nothing. Thread-safe. */
fe_status fe_serve_submit_n(fe_ctx *ctx, const fe_request *reqs, int n, uint64_t *tickets);
/* Release several finished requests at once. All or nothing: an unknown,
   unfinished or repeated ticket releases none (FE_ERR_INVALID_ARG). Thread-safe. */
fe_status fe_serve_release_n(fe_ctx *ctx, const uint64_t *tickets, int n);
/* Completion queue. Waits up to timeout_us microseconds (0: do not wait) until at
   least one request has finished that this call has not yet returned, then writes
   up to `max` finished requests, in completion order, to tickets[] and results[]
   (host arrays of `max` entries) and their number to *n_out (0 on timeout). Each
   finished request is returned once; requests released before they are returned
   are skipped. Results are as fe_serve_poll's; the outputs stay valid until
   fe_serve_release. Thread-safe; a request is returned to exactly one caller. */
fe_status fe_serve_wait_any(fe_ctx *ctx, int64_t timeout_us, uint64_t *tickets, fe_result *results, int max,
                            int *n_out);

/* Number of kernels this library has launched in this process (graph replays
   count the kernels in the graph). */
uint64_t fe_launch_count(void);

/* Failure-detection self-test (no counterpart in the paper): launches one block
   whose bounded wait on a bulk-copy barrier cannot complete (no copy is issued),
   with `polls` poll iterations (1..2^22, about 0.3 us each), then reports the
   device status like fe_ctx_sync. Expected: FE_ERR_TIMEOUT, after which the
   context remains usable; any other result means the detection is broken. */
fe_status fe_selftest_bounded_wait(fe_ctx *ctx, unsigned polls, void *stream);

/* Fault injection on the host, for tests of failure detection (no counterpart in
   the paper). Nothing is made to fault, trap or hang on the GPU:
   FE_FAULT_ALLOC       the next `count` device allocations of this context
                        (scratch growth, staging buffers, resident meshes, batch
                        plans, served outputs) fail as out of memory without
                        calling the allocator; the entry point that needed one
                        returns FE_ERR_OOM (a served request finishes with it) and
                        the context stays usable. `param` is ignored.
   FE_FAULT_SKIP_TILES  the next `count` main-kernel launches of fe_integrate_tet
                        and fe_integrate_prism (tiled kernels, one or two threads
                        per element) skip every tile whose index is a multiple of
                        `param` (>= 1): its elements are neither read nor
                        written, and a status bit makes the next fe_ctx_sync
                        return FE_ERR_PARTIAL.
   FE_FAULT_NONE        clears both.
   FE_ERR_INVALID_ARG for a null context, count < 0, param < 1 with
   FE_FAULT_SKIP_TILES or an unknown kind. */
typedef enum fe_fault { FE_FAULT_NONE = 0, FE_FAULT_ALLOC = 1, FE_FAULT_SKIP_TILES = 2 } fe_fault;
fe_status fe_ctx_inject_fault(fe_ctx *ctx, fe_fault kind, int64_t count, int64_t param);

/* Self-test of the double multiplications and additions that the FP64 kernels
   run in integer instructions (no counterpart in the paper; a test of the
   implementation): the same inputs through the integer-instruction operations
   (out_int) and the double-precision instructions (out_hw), which must agree bit
   for bit. Device arrays on the current device; enqueued on `stream`, returns
   after it finishes.
     what = 0: x, y operands [n]; out [2n]: the n products, then the n sums.
     what = 1: generic tetrahedra, TET4, per-element coefficients: x coordinates
               [n][4][3], y coefficients [n][20]; out [n][20]: A^e (16) then b^e.
     what = 2: Laplace tetrahedra, TET1: x as above, y d^0 [n]; out as above.
     what = 3: x, y operands [n]; out [n]: the products by the form that leaves
               special cases to its caller, completed there by the DMUL
               instruction (the kernels redo such an element on the double pipe).
     what = 4: as 3 for the sums (the addition that leaves special cases to its
               caller, completed by the DADD instruction).
   In 1 and 2 the integer-instruction side redoes an element on the double pipe
   when a multiplication or an addition meets a special case, as the kernels do.
   Degenerate elements give zeros. FE_ERR_INVALID_ARG for a bad `what`, n < 0 or
   null arrays. */
fe_status fe_selftest_f64_int(int what, const double *x, const double *y, int64_t n, double *out_int,
                              double *out_hw, void *stream);

/* Profiling: when on, the integration calls record CUDA events around their main
   kernel on the launching stream; fe_ctx_kernel_time returns the summed device
   time in ms and the launch count since the last reset (it synchronises). */
fe_status fe_ctx_set_profiling(fe_ctx *ctx, int on);
fe_status fe_ctx_kernel_time(fe_ctx *ctx, double *ms, int64_t *launches, int reset);

/* Autotuner: time every candidate launch shape for the key of (type, args, out)
   now, on these buffers, and keep the fastest. Candidates: blocks of 64 threads
   up to the kernel's limit (powers of two), persistent or not, and with
   element-contiguous coordinates and outputs, coefficient arrays and the QSS
   order, several threads per element (the intra-element parallelism of Sec. 3.3,
   Algorithms 4 and 5, with the QSS loop order kept):
     2 per prism: each thread takes the three points of one zeta level of
       Algorithm 2's point loop and the pair adds its partial results;
     4 per tetrahedron: one row of A^e and one entry of b^e per thread, the
       Jacobian terms formed once per element and shared by shuffles;
     6 per prism: thread q forms the Jacobian terms at point q, passes them to the
       group by shuffles and owns row q of A^e and entry q of b^e;
     16 per tetrahedron (the entry per work-item of the entry-outer orderings,
       Algorithm 7): thread 4 r + s delivers entry (r, s) of A^e (and b^e_r when
       s = 0), the Jacobian terms formed once per element and shared by shuffles.
   Writes the tuning cache if set. */
fe_status fe_tune(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                  void *stream);
/* Pin the launch shape of a key (threads = elements per block: 32..512 for
   tetrahedra, 32..256 for prisms, a multiple of 32; persistent 0 or 1), as the
   autotuner would; FE_ERR_UNSUPPORTED if its shared memory does not fit. */
fe_status fe_set_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                       int block_threads, int persistent);
/* The launch shape that the next call with this key would use: threads per
   block (elements per block x threads per element, in whole warps of groups as
   fe_set_launch_shape describes), and whether the grid is persistent (one wave
   of resident blocks striding over tiles) or one block per tile. */
fe_status fe_get_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                       int *block_threads, int *persistent);

/* Launch shape with the threads per element made explicit. */
typedef struct fe_launch_shape {
    int elems_per_block;           /* elements per tile (one block per tile) */
    int threads_per_elem;          /* 1; 2 or 6 (prisms), 4 or 16 (tetrahedra), as described at fe_tune */
    int persistent;                /* 0 or 1 */
} fe_launch_shape;
/* As fe_get_shape / fe_set_shape. Set: a warp holds 32 / threads_per_elem
   elements (5 with 6 threads per element, two lanes idle), so elems_per_block
   must be a multiple of that, and the block's threads (elems_per_block /
   (32 / threads_per_elem) x 32) at most the kernel's limit (512 for tetrahedra
   with one thread per element in the FP64 and mixed forms, 256 otherwise);
   FE_ERR_INVALID_ARG otherwise. FE_ERR_UNSUPPORTED for several threads per
   element where the key does not allow it (fe_tune), or if the shared memory does
   not fit. */
fe_status fe_get_launch_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                              fe_launch_shape *shape);
fe_status fe_set_launch_shape(fe_ctx *ctx, fe_elem_type type, const fe_elem_args *args, const fe_out *out,
                              const fe_launch_shape *shape);
/* Pin the shape of batch plans built from now on (fe_batch_submit of a new item
   list): elems_per_block (32..256, a multiple of 32) elements per tile for every
   combination, threads_per_elem (1 or 2) threads per prism element, at most 256
   threads per block; persistent 1 (counter-driven persistent grids) or 0 (one
   block per tile).
   NULL returns to tuned (autotune on) or default shapes. Lists already submitted
   keep their plans for the shape they were built with. */
fe_status fe_batch_set_shape(fe_ctx *ctx, const fe_launch_shape *shape);

/*
 * Mixed-precision tetrahedron integration that allocates nothing (the paper has
 * no counterpart; it is a service to callers that cannot call cudaMalloc, such
 * as code running inside a device-memory arena owned by a host application,
 * real-time loops that forbid allocator calls, or plugins that may not create a
 * context of this library).
 * Same inputs, outputs, layouts and results as fe_integrate_tet with
 * prec = FE_FP32_MIXED and device buffers (SOA or AOS coordinates); no context.
 * A node table, packed output, the coefficient function and the SQS / SSQ
 * orderings are rejected with FE_ERR_UNSUPPORTED. Its scratch (the list of
 * elements sent to the double-precision Jacobian pass, a counter and a status
 * word) is a fixed 4 MiB array in the library's device image, which every GPU
 * that loads the library holds until the process exits. Hence at most 524,256
 * elements per call; larger n_elem is rejected with FE_ERR_INVALID_ARG before any
 * GPU work. Runs on the calling thread's current device. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress); make that
 * first call before any stream capture. The address is kept for the life of the
 * process: calls after a device reset (cudaDeviceReset) are not supported. Every call clears the counter and the
 * status word, launches its two kernels on `stream` and returns after they
 * finish, reporting FE_ERR_TIMEOUT if a bulk-copy wait ran out. All calls share
 * the array: calls that overlap on the GPU (other streams or threads at the same
 * time) race and must not be made. Calls no cudaMalloc, cudaFree or other
 * allocating routine.
 */
fe_status fe_integrate_tet_noalloc(const fe_elem_args *args, const fe_out *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FE_H_ */
