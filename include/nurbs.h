/*
 * libnurbs -- GB300 (sm_103a) kernels for the data-parallel hot path of NURBS-Diff
 * (Prasad et al., arXiv 2104.14547): batched evaluation of rational B-spline
 * curves and surfaces on sample grids and its backward pass.
 *
 * Conventions for every entry point below
 * ---------------------------------------
 * - Pointers named d_* (and every float array argument of an execution call) are
 *   DEVICE pointers owned by the caller; h_* are host pointers.  The library never
 *   frees or retains caller memory beyond the call, and execution calls allocate
 *   no device memory: all scratch lives in a caller-provided workspace.
 * - Execution calls are asynchronous on the given stream (a cudaStream_t; NULL is
 *   the legacy default stream).  They return after the launch; device-side data
 *   errors are reported through nurbs_plan_get_error().
 * - All arithmetic is FP32.  Layouts are row-major, u the slow index.
 * - Calls sharing one workspace must not overlap on the GPU (they share counters
 *   and partial-sum slots).
 *
 * Data layout (packed, ragged batch)
 * ----------------------------------
 *   knots[]   float   each item's U (n1+p+1 floats) and V (m1+q+1) at desc offsets
 *   ctrl[]    float4  each item's control net [n1][m1] of (x, y, z, w): the
 *                     Cartesian control point P_ij and its weight w_ij (Eq. 3);
 *                     the offset must make the address 16-byte aligned
 *   params[]  float   each item's u samples (nu) and v samples (nv),
 *                     non-decreasing, inside [U_p, U_{n+1}] and [V_q, V_{m+1}]
 *   pts[]     float   each item's output block [nu][nv][3] at desc.pts * 3
 * Gradients use the layouts of the arrays they differentiate: grad_ctrl[] is a
 * float4 array (dL/dx, dL/dy, dL/dz, dL/dw) at the ctrl offsets; grad_knots[] is
 * a float array at the knot offsets.
 * A curve is an item with one parametric direction: p = its degree, n1 = its
 * control-point count, nu = its sample count; q, m1, nv, knot_v and param_v are
 * ignored.  Its output block is [nu][3].
 */
#ifndef NURBS_H
#define NURBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t. */
typedef struct CUstream_st* nurbs_stream_t;

typedef enum nurbs_status {
    NURBS_OK = 0,
    NURBS_ERR_ARG = 1,          /* NULL pointer, negative or zero size, bad kind / flag */
    NURBS_ERR_KNOTS = 2,        /* device check: knots decreasing, or first/last span empty */
    NURBS_ERR_DEGREE = 3,       /* degree outside [1, NURBS_MAX_DEGREE] or fewer than p+1 control points */
    NURBS_ERR_DOMAIN = 4,       /* device check: a sample outside [U_p, U_{n+1}] */
    NURBS_ERR_ORDER = 5,        /* device check: samples not non-decreasing */
    NURBS_ERR_WORKSPACE = 6,    /* workspace NULL, too small, misaligned, or plan not bound */
    NURBS_ERR_CUDA = 7,         /* a CUDA runtime call failed (see nurbs_last_cuda_error) */
    NURBS_ERR_SIZE = 8,         /* an item exceeds a kernel limit (control net, offsets) */
    NURBS_ERR_KIND = 9          /* the plan was built for the other kind (curve vs surface) */
} nurbs_status;

#define NURBS_MAX_DEGREE 5
#define NURBS_MAX_CTRL 4096     /* control points per direction */

enum { NURBS_KIND_SURFACE = 0, NURBS_KIND_CURVE = 1 };

/* One item (surface or curve) of a packed batch.  Offsets are element offsets
 * into the arrays named in the layout note above. */
typedef struct nurbs_desc {
    int32_t p, q;        /* degrees */
    int32_t n1, m1;      /* control points per direction (n+1, m+1) */
    int32_t nu, nv;      /* sample counts per direction */
    int32_t adam_step;   /* nurbs_fit_step: this item's 1-based Adam step (0 = the call's step) */
    float grad_scale;    /* nurbs_mse_fwd_bwd / nurbs_fit_step / nurbs_mse_fwd_bwd_noalloc: this
                            item's own scale of dL/dS = grad_scale * (S - T); 0 = the call's
                            grad_scale.  2 / (3 nu nv) makes the item's loss the mean over its
                            own points (Sec. 4, Eq. 12), so its gradient does not depend on the
                            other items of the batch.  Negative or non-finite: NURBS_ERR_ARG. */
    int64_t knot_u;      /* offset of U in knots[] (floats) */
    int64_t knot_v;      /* offset of V in knots[] (floats) */
    int64_t ctrl;        /* offset of the control net in ctrl[] (float4 elements) */
    int64_t param_u;     /* offset of the u samples in params[] (floats) */
    int64_t param_v;     /* offset of the v samples in params[] (floats) */
    int64_t pts;         /* offset of the output block in pts[] (points, 3 floats each) */
} nurbs_desc;

/* Tile shape for a plan.  Zero fields take the library's defaults. */
typedef struct nurbs_tile_cfg {
    int32_t rows;        /* sample rows per tile (surfaces; curves use one row) */
    int32_t warps;       /* warps per CTA (1..8; default 8) */
    int32_t ctas_per_sm; /* persistent CTAs per SM (0 = as many as fit).  k >= 2 also sizes the
                            shared memory of the gradient kernels so that k CTAs fit on an SM:
                            single-tile items whose adjoint no longer fits in shared memory
                            reduce it through the workspace, then no staged control net.
                            Results are the same. */
    int32_t max_ctas;    /* cap on the CTAs of each launch (0 = none); lets plans share the GPU */
} nurbs_tile_cfg;

/* Adam hyper-parameters (Kingma & Ba; the optimiser of Sec. 4). */
typedef struct nurbs_adam {
    float lr, beta1, beta2, eps;
} nurbs_adam;

typedef struct nurbs_plan nurbs_plan;

/*
 * nurbs_plan_create -- split a batch into tiles (host only, no GPU work).
 *   kind      NURBS_KIND_SURFACE or NURBS_KIND_CURVE
 *   h_desc    host array of `count` descriptors (copied; may be freed afterwards)
 *   cfg       tile shape, or NULL for defaults
 *   out       receives the plan; release with nurbs_plan_destroy
 * Errors: NURBS_ERR_ARG, NURBS_ERR_DEGREE, NURBS_ERR_SIZE.  Sizes only are
 * checked here; knot and sample values are checked on the device.
 */
nurbs_status nurbs_plan_create(int32_t kind, const nurbs_desc* h_desc, int32_t count,
                               const nurbs_tile_cfg* cfg, nurbs_plan** out);

/* Bytes of device workspace the plan needs (256-byte aligned pointer required). */
size_t nurbs_plan_workspace_size(const nurbs_plan* plan);

/* Points (samples) the plan evaluates, summed over items. */
int64_t nurbs_plan_points(const nurbs_plan* plan);

/* Tiles the plan launches and the CTAs of one launch (for reporting). */
int32_t nurbs_plan_tiles(const nurbs_plan* plan);
int32_t nurbs_plan_ctas(const nurbs_plan* plan);

/*
 * nurbs_plan_occupancy -- resident CTAs per SM of the plan's kernels for launch
 * kind `op` (the fewest over its degree groups) and the largest dynamic shared
 * memory of one CTA, in bytes (smem_bytes may be NULL).  op: 0 forward,
 * 1 backward, 2 backward with knot gradients, 3 MSE step, 4 MSE step with knot
 * gradients (also the fit step), 5 forward with tangents.  Lets a caller that
 * runs several plans side by side size their CTA caps (nurbs_tile_cfg.max_ctas)
 * by what really fits on an SM.  Queries the current device.
 * Errors: NURBS_ERR_ARG, NURBS_ERR_SIZE (a kernel cannot hold the plan's tile),
 * NURBS_ERR_CUDA.
 */
nurbs_status nurbs_plan_occupancy(const nurbs_plan* plan, int32_t op, int32_t* ctas_per_sm, int32_t* smem_bytes);

/*
 * nurbs_plan_bind -- attach a device workspace to the plan: uploads the item and
 * tile tables and zeroes the counters and the error word (async on `stream`; the
 * host tables are staged in plan-owned host memory that stays valid until the
 * plan is destroyed).  Must precede any execution call with this plan, and be
 * repeated if the workspace pointer changes.
 * Errors: NURBS_ERR_ARG, NURBS_ERR_WORKSPACE, NURBS_ERR_CUDA.
 */
nurbs_status nurbs_plan_bind(nurbs_plan* plan, void* d_workspace, size_t bytes, nurbs_stream_t stream);

void nurbs_plan_destroy(nurbs_plan* plan);

/*
 * nurbs_plan_set_knot_sigma -- choose the knot derivative of later backward,
 * MSE and fit-step calls on this plan (host only).
 *   sigma == 0 (the default): the exact almost-everywhere derivative of Eq. 4,
 *     i.e. the degree-0 indicators' knot derivative taken as 0 (the sigma -> 0
 *     limit of Sec. 3.2).
 *   sigma > 0: the paper's Gaussian-smoothed indicator.  The degree-0 function
 *     N^0_j gets the knot derivative -G(u - U_j) at U_j and +G(u - U_{j+1}) at
 *     U_{j+1}, with G(x) = exp(-x^2 / 2 sigma^2) / (sigma sqrt(2 pi)).  These
 *     terms are pushed through the Cox-de Boor triangle, and each sample adds
 *     them for the 2p knots it already touches.  The knots one step further out
 *     lie at least p spans away and are left out.
 * The end knots still get 0.  Errors: NURBS_ERR_ARG for a negative or
 * non-finite sigma.
 */
nurbs_status nurbs_plan_set_knot_sigma(nurbs_plan* plan, float sigma);

/*
 * nurbs_plan_set_grad_homogeneous -- choose the parameterisation of the control
 * point gradients that later backward, MSE and fit-step calls on this plan write
 * to grad_ctrl (host only).
 *   on == 0 (the default): the paper's parameters, (dL/dx, dL/dy, dL/dz, dL/dw)
 *     for the Cartesian point P and its weight w (Eq. 7, Eq. 8).
 *   on == 1: the homogeneous point Pw = (w x, w y, w z, w) of Eq. 3,
 *     (dL/dPw.x, dL/dPw.y, dL/dPw.z, dL/dPw.w), related to the above by
 *     dL/dPw.xyz = (dL/dP) / w and dL/dPw.w = dL/dw - P . (dL/dP) / w.
 * nurbs_fit_step's Adam update always acts on (P, w).  Errors: NURBS_ERR_ARG for
 * a null plan or `on` outside {0, 1}.
 */
nurbs_status nurbs_plan_set_grad_homogeneous(nurbs_plan* plan, int32_t on);

/*
 * nurbs_plan_get_error -- synchronise `stream`, read and clear the device error
 * word written by the device-side checks of earlier calls.  *flags receives the
 * raw bit set (bit k set <=> status k was raised); returns the lowest raised
 * status, or NURBS_OK.
 */
nurbs_status nurbs_plan_get_error(nurbs_plan* plan, nurbs_stream_t stream, uint32_t* flags);

/*
 * nurbs_eval_surface -- forward evaluation of every surface item (Eq. 3,
 * Sec. 3.1 steps 1-3, Alg. 1): span search, nonzero Cox-de Boor basis (Eq. 4),
 * homogeneous weighted sum and perspective divide, S(u_a, v_b) -> pts.
 */
nurbs_status nurbs_eval_surface(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                const float* params, float* pts, nurbs_stream_t stream);

/* nurbs_eval_curve -- the same for curve items (Sec. 3, curves). */
nurbs_status nurbs_eval_curve(const nurbs_plan* plan, const float* knots, const float* ctrl,
                              const float* params, float* pts, nurbs_stream_t stream);

/*
 * nurbs_eval_surface_derivs -- forward evaluation with the surface tangents and
 * unit normals that the paper's surface-offsetting application needs (the
 * derivatives S_,u and S_,v of Sec. 3.2; offsetting in Sec. 4).
 *   Tangents: S_u = (A_u - W_u S) / W, where S' = (A, W) is the homogeneous point
 *   of Eq. 3 and A_u, W_u take the u-derivative of the basis (of Eq. 4) in place
 *   of the basis.  S_v is defined the same way.
 *   Normals: S_u x S_v / |S_u x S_v|; a degenerate point (zero cross product)
 *   gets 0.
 * pts, du, dv, normals: device arrays in the points' layout ([npts][3] floats at
 * each item's pts offset).  Any of them may be NULL, but not all.  Samples on a
 * knot see the derivative from the right, except at the end of the domain.
 * Errors: as nurbs_eval_surface; NURBS_ERR_ARG when every output is NULL.
 */
nurbs_status nurbs_eval_surface_derivs(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                       const float* params, float* pts, float* du, float* dv, float* normals,
                                       nurbs_stream_t stream);

/*
 * nurbs_eval_curve_derivs -- curve points and tangents C'(u) = (A' - W' C) / W
 * (the curve form of nurbs_eval_surface_derivs).  pts and tangents are device
 * arrays in the points' layout.  Either may be NULL, but not both.
 */
nurbs_status nurbs_eval_curve_derivs(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                     const float* params, float* pts, float* tangents, nurbs_stream_t stream);

/*
 * nurbs_backward -- vector-Jacobian product of the evaluation (Sec. 3.2, Eq. 7,
 * Eq. 8, Eq. 9, the knot derivative, Alg. 2), for surface or curve plans.
 *   grad_pts    dL/dS in the pts layout
 *   grad_ctrl   receives (dL/dx, dL/dy, dL/dz, dL/dw) per control point (or the
 *               homogeneous form, see nurbs_plan_set_grad_homogeneous), or NULL
 *   grad_knots  receives dL/dU (and dL/dV), or NULL.  Knot gradients are the
 *               almost-everywhere derivative of the Cox-de Boor recursion (the
 *               sigma -> 0 limit of the smoothed indicator of Sec. 3.2); the
 *               p+1 knots at each end of a knot vector receive 0.
 * Outputs are overwritten, not accumulated.  Basis values are recomputed, not
 * stored by the forward call.
 */
nurbs_status nurbs_backward(const nurbs_plan* plan, const float* knots, const float* ctrl,
                            const float* params, const float* grad_pts, float* grad_ctrl,
                            float* grad_knots, nurbs_stream_t stream);

/*
 * nurbs_mse_fwd_bwd -- forward, MSE loss against `target` (pts layout) and the
 * backward of that loss in one launch (the L2 loss of Sec. 4 read as a mean
 * squared error, Eq. 1 chain rule).
 *   pts         receives S, or NULL to skip the write
 *   loss_items  receives each item's sum of squared differences (float[count]), or NULL
 *   grad_scale  dL/dS = grad_scale * (S - T) for items whose descriptor has
 *               grad_scale == 0; 2 / (3 * total points) gives the gradient of the
 *               mean over all coordinates of the batch.  An item with its own
 *               descriptor grad_scale > 0 uses that instead (per-item mean loss).
 * grad_ctrl / grad_knots as in nurbs_backward (either may be NULL).
 */
nurbs_status nurbs_mse_fwd_bwd(const nurbs_plan* plan, const float* knots, const float* ctrl,
                               const float* params, const float* target, float* pts,
                               float* grad_ctrl, float* grad_knots, float* loss_items,
                               float grad_scale, nurbs_stream_t stream);

/*
 * nurbs_fit_step -- one fused fitting step: forward, MSE against `target`,
 * backward, and an Adam update (Sec. 4, Eq. 13 with Adam) of every control point
 * and weight in place.  Knots are not updated.
 *   ctrl        control nets, updated in place
 *   adam_m/v    Adam moments, float4 per control point in the ctrl layout (zero
 *               before the first step), updated in place
 *   step        1-based Adam step number (bias correction) for items whose
 *               descriptor has adam_step == 0; other items use their own
 *   pts, loss_items, grad_knots  as in nurbs_mse_fwd_bwd (NULL to skip)
 */
nurbs_status nurbs_fit_step(const nurbs_plan* plan, const float* knots, float* ctrl,
                            const float* params, const float* target, float* pts,
                            float* adam_m, float* adam_v, const nurbs_adam* hp, int32_t step,
                            float grad_scale, float* loss_items, float* grad_knots,
                            nurbs_stream_t stream);

/*
 * nurbs_mse_fwd_bwd_noalloc -- the computation of nurbs_mse_fwd_bwd (same
 * arguments, same results) for callers that cannot allocate device memory: for
 * example a plug-in whose host application owns every device allocation, or code
 * running where cudaMalloc is not allowed (inside a host callback, or in a process
 * whose memory budget is fixed at start-up).  The paper has no counterpart; this
 * entry point exists only for such integrations.
 *   - It allocates nothing.  Its scratch is one fixed array of
 *     NURBS_NOALLOC_SCRATCH_BYTES bytes in the library's device image; every GPU
 *     that loads the library holds that array until the process exits.
 *   - The plan needs no workspace and no nurbs_plan_bind.  A plan whose
 *     nurbs_plan_workspace_size() exceeds NURBS_NOALLOC_SCRATCH_BYTES is rejected
 *     with NURBS_ERR_WORKSPACE before any GPU work.
 *   - All calls share the array: each call uploads the plan's tables into it and
 *     clears its counters first, and calls that overlap on the GPU (other streams,
 *     other host threads) race on it and give wrong results.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current).  Make that first call on each device
 *     before any stream capture begins.
 *   - Device-side data errors (knots, domain, sample order) go to an error word
 *     at the head of the array, which calls do not clear: it collects the checks
 *     of every call until nurbs_noalloc_get_error reads it.  nurbs_plan_get_error
 *     does not see them (it reads a plan's bound workspace).
 */
#define NURBS_NOALLOC_SCRATCH_BYTES (8u << 20)

nurbs_status nurbs_mse_fwd_bwd_noalloc(const nurbs_plan* plan, const float* knots, const float* ctrl,
                                       const float* params, const float* target, float* pts,
                                       float* grad_ctrl, float* grad_knots, float* loss_items,
                                       float grad_scale, nurbs_stream_t stream);

/*
 * nurbs_noalloc_get_error -- the nurbs_plan_get_error of nurbs_mse_fwd_bwd_noalloc
 * (no counterpart in the paper either): synchronise `stream`, read and clear the
 * error word of the allocation-free entry point's fixed array on the current
 * device.  *flags (may be NULL) receives the raw bit set collected by every
 * allocation-free call since the last read; returns the lowest raised status, or
 * NURBS_OK.  Allocates nothing.  Errors: NURBS_ERR_CUDA.
 */
nurbs_status nurbs_noalloc_get_error(nurbs_stream_t stream, uint32_t* flags);


/*
 * nurbs_chamfer -- the paper's point-set losses (Sec. 4) over `count` pairs of
 * point sets, with their gradients with respect to the first set.  Pair k has
 * points P[p_off[k] .. p_off[k+1]) and Q[q_off[k] .. q_off[k+1]):
 *   L_CD = sum_i min_j |P_i - Q_j| + sum_j min_i |P_i - Q_j|      (Chamfer)
 *   L_HD = max_i min_j |P_i - Q_j| + max_j min_i |P_i - Q_j|      (Hausdorff)
 * All arrays are device arrays.
 *   P, Q                points, [n][3] floats.
 *   p_off, q_off        int64 offsets in points, count+1 of them, non-decreasing.
 *   max_p, max_q        host bounds on the largest set of each side (grid size);
 *                       points beyond them are not processed.
 *   nn_p, dist_p        outputs, one per point of P: pair-local index of the
 *                       nearest Q point (-1 if the pair's Q is empty) and the
 *                       distance to it.  nn_q, dist_q: the same for Q.
 *   cd, hd              optional outputs, one per pair.
 *   grad_cd, grad_hd    optional outputs, [n][3] like P: gradients of L_CD and L_HD.
 *   scratch             optional: 2*total_p + total_q int32 of device scratch
 *                       (total_p = p_off[count], total_q = q_off[count]).  With it,
 *                       the Chamfer gradient buckets the Q points by nearest P point
 *                       (O(n + m) per pair).  Without it, each P point scans its
 *                       pair's whole nearest-point map (O(n m)).  The results are
 *                       the same.
 * Nearest points are decided on float32 squared distances, each rounded as
 * ((dx dx + dy dy) + dz dz); ties go to the first index.  A zero distance
 * contributes no gradient.  A pair with an empty side gives 0 and zero
 * gradients.  Asynchronous on `stream`; no allocation; deterministic.
 * Errors: NURBS_ERR_ARG (negative sizes, a missing required array),
 * NURBS_ERR_SIZE (count > 65535), NURBS_ERR_CUDA.
 */
nurbs_status nurbs_chamfer(int32_t count, const int64_t* p_off, const int64_t* q_off, int32_t max_p, int32_t max_q,
                           const float* P, const float* Q, int32_t* nn_p, float* dist_p, int32_t* nn_q,
                           float* dist_q, float* cd, float* hd, float* grad_cd, float* grad_hd,
                           int32_t* scratch, int64_t total_p, int64_t total_q, nurbs_stream_t stream);

/* Human-readable name of a status code (static string). */
const char* nurbs_status_string(nurbs_status status);

/* The last CUDA runtime error code seen by the library on this thread (0 = none). */
int32_t nurbs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NURBS_H */
