/*
 * wq.h -- C ABI of libwq: row-wise assembly of isogeometric mass and
 * stiffness matrices with weighted Gaussian quadrature on GB300 (sm_103a).
 *
 * Method (Barton, Puzyrev, Deng, Calo, "Efficient mass and stiffness matrix
 * assembly via weighted Gaussian quadrature rules for B-splines"):
 *   - uniform open knot vectors of maximal continuity per direction
 *     (Sec. 2.2, Eq. 3), degree p in {2, 3}, dimension d in {2, 3};
 *   - row i of the mass matrix M (Eq. Mass) and of the stiffness matrix K
 *     (Eq. Stiffness) is integrated by its own quadrature rule, Gaussian with
 *     respect to B_i (mass, Sec. 3.1, Eq. GaussQuadSys) or B_i' (stiffness,
 *     Sec. 3.2, Eq. GaussQuadSysStiff): p+1 nodes per direction, one per
 *     element of supp B_i; rows whose weight function touches the boundary
 *     use Gauss-Legendre on each element of the support (Remark closing
 *     Sec. 3);
 *   - the multivariate rule is the tensor product of the 1D rules (Eq.
 *     Decompo) and is applied by sum factorisation, one direction at a time,
 *     into the row's (2p+1)^d band (caption of Fig. 1).
 *
 * Inputs follow the problem statement of Sec. 2: degree and element counts
 * (uniform knots), a geometry map (Eq. Gmap1) restricted to separable maps
 * x_a = sum_i g_{a,i} B_i(xhat_a), and a coefficient field c multiplying the
 * integrands (c = 1 in Eq. Mass / Eq. Stiffness), given as a degree-3 spline
 * on the same mesh.  Only the diagonal metric terms have a weighted rule in
 * the paper (Sec. 3.2), which is why these calls take separable maps; maps
 * given by a full control net go through wq_assemble_general, which adds
 * mixed-derivative rules for the off-diagonal terms.
 *
 * Band layout (output): rows r = r1 + n1*(r2 + n2*r3) with n_a = nel_a + p,
 * each row holding (2p+1)^d entries; entry index
 *   (d3+p)*(2p+1)^2 + (d2+p)*(2p+1) + (d1+p)   for column s_a = r_a + d_a,
 * set to zero where a column index falls outside [0, n_a).
 *
 * Conventions for every entry point:
 *   - return value: a wq_status; no C++ exception, exit() or device trap
 *     crosses this boundary;
 *   - "device" pointers are CUDA device memory on the current device, owned
 *     by the caller; "host" pointers are ordinary host memory;
 *   - calls that take a stream enqueue asynchronous work on it (a CUDA
 *     stream handle, NULL = legacy default stream) and return once it is
 *     enqueued; problems the GPU detects (a Jacobian entry <= 0, a
 *     non-finite input) are reported by wq_status_check;
 *   - a wq_rules object owns device tables and a small per-call scratch
 *     area; calls that use the same wq_rules on different streams must not
 *     overlap in time.
 */
#ifndef WQ_H
#define WQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum wq_status {
  WQ_OK = 0,
  WQ_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, range) */
  WQ_ERR_UNSUPPORTED = 2,    /* degree/dimension outside {2,3}, too many elements */
  WQ_ERR_NO_CONVERGENCE = 3, /* a 1D rule failed its Newton solve or exactness check */
  WQ_ERR_GEOMETRY = 4,       /* some J_aa <= 0 at a quadrature point (folded map); the
                                result is still written with |J_aa| as in Eq. Mass */
  WQ_ERR_NONFINITE = 5,      /* NaN or Inf in the geometry or coefficients */
  WQ_ERR_CUDA = 6,           /* a CUDA runtime call failed */
  WQ_ERR_OOM = 7,            /* device allocation failed */
  WQ_ERR_TIMEOUT = 8,        /* reserved: a bounded device wait expired */
  WQ_ERR_CHECK = 9           /* a device-side range check failed: only libraries built with
                                -DWQ_CHECKED=1 run these checks; the access was skipped */
} wq_status;

typedef enum wq_precision {
  WQ_FP64 = 0,  /* FP64 throughout; band written as double */
  WQ_MIXED = 1, /* Jacobian and rule tables in FP64, contractions in FP32;
                   band written as float */
  WQ_DF64 = 2   /* Jacobian and rule tables in FP64, contractions in
                   double-float arithmetic (pairs of floats, ~48-bit
                   significand) on the FP32 pipe; band written as double.
                   Agrees with WQ_FP64 to ~1e-14 relative for inputs within
                   float's exponent range (|values| in 1e-30 .. 1e30) */
} wq_precision;

/* Kinds of 1D rules.  MASS and STIFFNESS are the rules of Sec. 3.1 and 3.2
 * (weight B_r with tests B_s; weight B_r' with tests B_s').  The two mixed
 * kinds integrate the off-diagonal metric terms of a non-separable map
 * (wq_assemble_general): MIXED_DW the weight B_r' with the tests B_s,
 * MIXED_WD the weight B_r with the tests B_s'. */
enum { WQ_KIND_MASS = 0, WQ_KIND_STIFFNESS = 1, WQ_KIND_MIXED_DW = 2, WQ_KIND_MIXED_WD = 3 };
enum {
  WQ_RULES_HOST_ONLY = 0,
  WQ_RULES_DEVICE = 1,
  /* Comparison rules (baselines; at most one, FP64 assembly only, no adjoint
   * or batch): every row with (p+1)-point Gauss-Legendre on each element of
   * its support (the element-wise Gauss point set), or the interior rows
   * with the Newton-Cotes-type weighted rules of Sec. 1 / Sec. 4 (nodes at
   * the knots and element midpoints of the support, 2p+1 per direction). */
  WQ_RULES_GAUSS_LEGENDRE = 2,
  WQ_RULES_NEWTON_COTES = 4,
  /* The weighted Gaussian rules for the boundary rows too (the Remark
   * closing Sec. 3: the systems "modified accordingly"): row r < p (and its
   * mirror image n-1-r) of each kind gets ceil(rank/2) nodes exact for the
   * products B_r^(nu) B_s^(nu) over every interacting s (rank r+p+1 for the
   * mass kind, r+p for the stiffness kind), with one more condition, on
   * B_r^(nu) (x/h)^(p-nu+1), when the rank is odd; defined for every mass
   * row and every stiffness row but p = 3 row 1, which keeps Gauss-Legendre,
   * as do all rows of directions with fewer than 2p+1 elements.  Assembly
   * calls only (mass, stiffness, both, host-buffer form): the apply, load,
   * adjoint, batch and no-alloc calls return WQ_ERR_UNSUPPORTED for it.  Not
   * combinable with the comparison rules. */
  WQ_RULES_BOUNDARY_WEIGHTED = 8
};

typedef struct wq_mesh {
  int dim;     /* 2 or 3 */
  int degree;  /* 2 or 3 */
  int nel[3];  /* elements per direction (entries beyond dim ignored), >= 1 */
} wq_mesh;

typedef struct wq_rules wq_rules; /* opaque */

/* Human-readable name of a status code (static storage). */
const char *wq_status_string(wq_status s);

/* Library version, major*10000 + minor*100 + patch. */
int wq_version(void);

/*
 * The univariate weighted Gaussian rule on the cardinal support [0, p+1]
 * (Sec. 3.1 for kind = WQ_KIND_MASS, Sec. 3.2 for kind = WQ_KIND_STIFFNESS):
 * writes p+1 nodes tau[k] (one per unit element, ascending) and weights
 * omega[k] (host arrays of length degree+1).  The rule satisfies
 * sum_k omega_k N(tau_k) N(tau_k - d) = int N(y) N(y - d) dy for d = -p..p
 * (N the cardinal B-spline, or its derivative for the stiffness kind).  The
 * free parameters are the paper's: tau_2 = 3/2 (p = 2), omega_1 = 1 and the
 * smaller tau_1 root (p = 3 stiffness).  Host only; returns
 * WQ_ERR_NO_CONVERGENCE if the solve or its exactness check fails.
 */
wq_status wq_rule_1d(int degree, int kind, double *tau, double *omega);

/*
 * Newton solve of the same rule from a caller-chosen start (host).  start
 * holds the unknowns of the symmetric rule: (tau_1, omega_1, omega_2) for
 * mass p=2, (tau_1, tau_2, omega_1, omega_2) for mass p=3, (tau_1, omega_1)
 * for stiffness p=2, (tau_1, tau_2, omega_2) for stiffness p=3.  Returns
 * WQ_ERR_NO_CONVERGENCE unless the iteration reaches a rule with one node in
 * each element that passes all 2p+1 exactness conditions (Sec. 3.1.2 shows
 * a start that does not).
 */
wq_status wq_rule_1d_from(int degree, int kind, const double *start, double *tau, double *omega);

/*
 * The mixed-derivative rules for the off-diagonal metric terms of a
 * non-separable map (Eq. Stiffness with a full Jacobian; the paper gives
 * rules for the diagonal pairs only, Sec. 3.2).  One node set on the
 * cardinal support [0, p+1] serves both mixed kinds: writes degree+1 nodes
 * y[k] (one per unit element, ascending, symmetric about (p+1)/2) and the
 * weights w[k] (antisymmetric) and v[k] (symmetric) such that, for
 * d = -p..p,
 *   sum_k w_k N(y_k - d)  = int N'(y) N(y - d) dy   (weight N', tests N),
 *   sum_k v_k N'(y_k - d) = int N(y) N'(y - d) dy   (weight N, tests N').
 * By the symmetries each kind has p independent conditions; p = 3 takes two
 * node pairs (six unknowns), p = 2 one pair and the centre node (four).
 * Host arrays of length degree+1; WQ_ERR_NO_CONVERGENCE if the Newton solve
 * or the exactness check fails.
 */
wq_status wq_rule_1d_mixed(int degree, double *y, double *w, double *v);

/*
 * Builds the per-direction row tables of a mesh: for every row of every
 * direction and both kinds, the rule points (interior rows: the weighted
 * Gaussian rule mapped to supp B_r; boundary rows: (p+1)-point
 * Gauss-Legendre on each element of supp B_r), the combined weights
 * W = h*omega*B_r^(nu)(x), and the values and derivatives of the p+1
 * B-splines acting at each point.  flags = WQ_RULES_DEVICE also allocates
 * and fills the device copy (current device) used by the assembly calls;
 * WQ_RULES_HOST_ONLY builds host tables only (no CUDA call is made).
 * *out receives a new object to be released with wq_rules_free.
 * WQ_ERR_OOM if the device allocation fails (also forced, before any CUDA
 * call, when the environment variable WQ_FAULT_DEVICE_ALLOC is set: a hook
 * for testing callers' error paths); nothing is leaked on any error.
 */
wq_status wq_rules_build(const wq_mesh *mesh, int flags, wq_rules **out);

/* Releases a wq_rules object and its device memory (NULL is ignored). */
void wq_rules_free(wq_rules *rules);

/*
 * Host view of one row's 1D rule: direction dir (0-based, < dim), kind
 * (WQ_KIND_*; the mixed kinds exist for rules objects of the weighted
 * Gaussian rules without other flags, else WQ_ERR_UNSUPPORTED; their
 * interior rows use wq_rule_1d_mixed mapped to supp B_r, W = w_k for
 * MIXED_DW and W = h v_k for MIXED_WD, their boundary rows Gauss-Legendre
 * with B_r' or B_r folded in), row index in [0, nel_dir + p).  *npts receives the point count (at most
 * degree*(degree+1) for the weighted rules, (degree+1)^2 with
 * WQ_RULES_GAUSS_LEGENDRE); x, w receive the points and combined weights W,
 * elem the element of each point, each with room for *npts values (call
 * with NULL arrays first to learn it).  Any output pointer may be NULL.
 */
wq_status wq_rules_row(const wq_rules *rules, int dir, int kind, int row, int *npts, double *x, double *w,
                       int *elem);

/* Sizes of a mesh: rows = prod(nel_a + p); band = (2p+1)^dim entries per row;
 * nnz = band entries with in-range columns (per matrix); coef = prod(nel_a + 3). */
int64_t wq_rows(const wq_rules *rules);
int64_t wq_band_width(const wq_rules *rules);
int64_t wq_band_nnz(const wq_rules *rules);
int64_t wq_coef_count(const wq_rules *rules);

/*
 * Algorithmic floating-point operation count of assembling rows
 * [row_begin, row_end) (mass if want_m, stiffness if want_k): the
 * multiply-adds of the sum-factorised contractions on the non-zero band
 * structure (2 flops each), excluding coefficient evaluation, which is
 * returned separately in *coef_flops (may be NULL).  Host only.
 */
double wq_flop_count(const wq_rules *rules, int want_m, int want_k, int64_t row_begin, int64_t row_end,
                     double *coef_flops);

/*
 * Assembly of rows [row_begin, row_end) (0 <= row_begin <= row_end <= rows)
 * into band arrays (Eq. Mass, Eq. Stiffness, weighted Gaussian rules):
 *   geom[a]  device, n_a = nel_a + p doubles: control values of x_a (host
 *            array of dim device pointers);
 *   coef     device, prod(nel_a + 3) doubles, x fastest: degree-3 spline of
 *            the coefficient c; NULL means c = 1;
 *   M, K     device, (row_end - row_begin) * band entries, double for
 *            WQ_FP64 and WQ_DF64, float for WQ_MIXED; row row_begin is stored first;
 *            may be NULL when row_begin == row_end (nothing is written).
 * wq_assemble_mass_stiffness writes both (the fused path); the single-matrix
 * forms write one.  The rules object must have been built with
 * WQ_RULES_DEVICE on the current device.  Output buffers must not overlap
 * the inputs.
 */
wq_status wq_assemble_mass(const wq_rules *rules, const double *const *geom, const double *coef,
                           wq_precision prec, void *M, int64_t row_begin, int64_t row_end, void *stream);
wq_status wq_assemble_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                wq_precision prec, void *K, int64_t row_begin, int64_t row_end, void *stream);
wq_status wq_assemble_mass_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                     wq_precision prec, void *M, void *K, int64_t row_begin, int64_t row_end,
                                     void *stream);

/*
 * The same assembly end to end between host buffers (Eq. Mass, Eq.
 * Stiffness; the computation of wq_assemble_mass_stiffness): the host
 * inputs are copied to caller-owned device buffers on `stream`, rows
 * [row_begin, row_end) are assembled in `nchunks` consecutive ranges into
 * caller-owned device bands, and each range's bands are copied to the host
 * on `copy_stream` while the next range is being assembled on `stream`.
 *   geom_host[a], coef_host  host inputs as for wq_assemble_mass_stiffness
 *                            (coef_host NULL: c = 1);
 *   geom_dev[a], coef_dev    device buffers of the same sizes, overwritten
 *                            (coef_dev unused, may be NULL, when coef_host
 *                            is NULL);
 *   M_dev, K_dev             device bands of (row_end - row_begin) rows
 *                            (double for WQ_FP64 and WQ_DF64, float for
 *                            WQ_MIXED), overwritten: the staging area;
 *   M_host, K_host           host bands of the same shape and type,
 *                            overwritten, row row_begin first;
 *   nchunks                  1 .. 1024 row ranges;
 *   stream, copy_stream      two different CUDA streams of the current device.
 * The call returns once everything is enqueued; `stream` then waits for the
 * last copy, so a synchronisation of `stream` makes M_host and K_host valid.
 * The host buffers must stay alive, and unread, until then; page-locked host
 * memory (cudaHostAlloc, cudaHostRegister) lets the copies overlap the
 * assembly, pageable memory makes them synchronous.  Two CUDA events are
 * created and released per call; no device memory is allocated.  Device-
 * detected problems are reported by wq_status_check, argument errors as for
 * wq_assemble_mass_stiffness (WQ_ERR_ARG also for nchunks out of range or
 * equal streams).
 */
wq_status wq_assemble_mass_stiffness_host(const wq_rules *rules, const double *const *geom_host,
                                          const double *coef_host, wq_precision prec, void *M_host, void *K_host,
                                          double *const *geom_dev, double *coef_dev, void *M_dev, void *K_dev,
                                          int64_t row_begin, int64_t row_end, int nchunks, void *stream,
                                          void *copy_stream);

/*
 * Assembly for a map given by its full control net (Eq. Gmap1): rows
 * [row_begin, row_end) of M (Eq. Mass) and K (Eq. Stiffness with the full
 * metric C = c |det J| J^-1 J^-T), in the band layout above.
 *   net   device, dim * prod(n_a) doubles (n_a = nel_a + p): component a of
 *         control point (i1, i2, i3) at net[a*prod(n) + i1 + n1*(i2 + n2*i3)];
 *   coef  device coefficient spline as for wq_assemble_mass_stiffness, or NULL;
 *   M, K  device bands of row_end - row_begin rows (double for WQ_FP64,
 *         float for WQ_MIXED); either (not both) may be NULL.
 * M uses the mass rule in every direction with the factor c |det J| at each
 * point; K is the sum over a, b of the terms dB_r/dxhat_a C_ab dB_s/dxhat_b,
 * each with the tensor product of the stiffness rule where d = a = b, the
 * mixed rule WQ_KIND_MIXED_DW where d = a != b, WQ_KIND_MIXED_WD where
 * d = b != a and the mass rule in the other directions; the factors are
 * evaluated at every point from the full Jacobian.  Boundary rows use
 * Gauss-Legendre in every kind.  Exact (up to rounding) for affine maps with
 * c = 1; for a separable net the result equals wq_assemble_mass_stiffness
 * up to rounding.  prec: WQ_FP64 (everything in FP64), or WQ_MIXED: the
 * Jacobian in FP32 from the net's scaled differences p (P_i - P_{i-1}) /
 * (t_{i+p} - t_i), formed in FP64 (each column of J is then a sum of the
 * degree p-1 derivative spline's terms, free of the cancellation of
 * sum_i P_i B_i'), and the metric and contractions in FP32, ~1e-7 relative;
 * WQ_DF64 gives WQ_ERR_UNSUPPORTED.  The rules object must be built with
 * WQ_RULES_DEVICE and no other flag (else WQ_ERR_UNSUPPORTED).  A Jacobian determinant <= 0 or a non-finite value
 * is reported by wq_status_check (WQ_ERR_GEOMETRY, WQ_ERR_NONFINITE; the
 * bands are written with |det J|).  The metric factors of a slab of rows
 * (and, for WQ_MIXED, the difference nets, dim^2 floats per control
 * point) are kept in a scratch array of the rules object (the factors at
 * most 1 GiB, or one x3 plane's points if more; the environment variable
 * WQ_GENERAL_SLAB_BYTES lowers that bound), allocated by the first call that needs it and
 * grown by later calls (synchronising `stream` first); WQ_ERR_OOM if that
 * allocation fails.
 */
wq_status wq_assemble_general(const wq_rules *rules, const double *net, const double *coef, wq_precision prec,
                              void *M, void *K, int64_t row_begin, int64_t row_end, void *stream);

/*
 * Matrix-free apply: y_M = M x and y_K = K x for rows [row_begin, row_end)
 * of the matrices of wq_assemble_mass_stiffness (Eq. Mass, Eq. Stiffness
 * with the weighted Gaussian rules; K x is the operator of Eq. LinSys), with
 * every band entry formed as in the assembly and multiplied into x at once:
 * the band is never stored.
 *   geom, coef  as for wq_assemble_mass_stiffness;
 *   x           device, one value per row of the whole mesh (wq_rows), in
 *               row order, double for WQ_FP64 and WQ_DF64, float for
 *               WQ_MIXED;
 *   yM, yK      device, row_end - row_begin values of the same type, row
 *               row_begin first; either (not both) may be NULL.
 * y_r is the sum over the row's band of entry times x at the entry's column,
 * in the precision of `prec` (double-float products and sums for WQ_DF64).
 * Rules objects built for the weighted Gaussian rules on the device
 * (WQ_RULES_DEVICE, no comparison-rule flag), 2D or 3D; comparison-rule
 * objects give WQ_ERR_UNSUPPORTED.  x must not overlap yM or yK.
 */
wq_status wq_apply_mass_stiffness(const wq_rules *rules, const double *const *geom, const double *coef,
                                  wq_precision prec, const void *x, void *yM, void *yK, int64_t row_begin,
                                  int64_t row_end, void *stream);

/*
 * Load vector (Eq. Load): b_r = integral of f B_r |det J| for rows
 * [row_begin, row_end), each row integrated by its own weighted Gaussian
 * mass rule.  Since the basis is a partition of unity, this is M(f) 1, the
 * mass matrix with coefficient f applied to the vector of ones, and is
 * computed that way by the apply kernels.
 *   geom   as for wq_assemble_mass_stiffness;
 *   f      device, prod(nel_a + 3) doubles, x fastest: degree-3 spline of
 *          the source f; NULL means f = 1;
 *   b      device, row_end - row_begin values, double for WQ_FP64 and
 *          WQ_DF64, float for WQ_MIXED.
 * Same rules-object requirements as wq_apply_mass_stiffness.
 */
wq_status wq_assemble_load(const wq_rules *rules, const double *const *geom, const double *f, wq_precision prec,
                           void *b, int64_t row_begin, int64_t row_end, void *stream);

/*
 * Adjoint of the assembly with respect to the coefficient spline: every band
 * entry of M and K (Eq. Mass, Eq. Stiffness with the weighted Gaussian rules)
 * is linear in the coefficients C of c, so for band weights G, H the
 * functional
 *   J(C) = sum over rows [row_begin, row_end) and band entries of
 *          G .* K(C) + H .* M(C)
 * has the gradient dJ/dC = A^T (G, H), A the linear map C -> (K, M) that the
 * forward calls apply.  This is the backward pass of the assembly.
 *   geom       as for wq_assemble_mass_stiffness;
 *   G, H       device band arrays laid out like K and M of those rows (double
 *              for WQ_FP64 and WQ_DF64, float for WQ_MIXED); either may be
 *              NULL (a zero weight);
 *   grad       device, prod(nel_a + 3) doubles, x fastest; overwritten.
 * Every partial result goes to its own slot of a scratch array and is summed
 * in a fixed order, never by atomics, so repeated calls on the same inputs
 * return the same bits: in 2D each chunk of rows writes its block of the
 * gradient and a second kernel adds, per coefficient, the blocks that touch
 * it; in 3D each chunk writes the gradient of its partial contractions
 * (Ubar), a second kernel takes the x2 and x3 stages per block of 8 lines of
 * a plane and 4 coefficient columns (summing the chunks of a column in chunk
 * order and the block's lines in line order), and a third adds the blocks
 * per coefficient.  The scratch belongs to the rules object (3D cubic: about
 * 180 values of the arithmetic type per row, 1.5 GB at 96^3 in FP64): the
 * first call that needs it allocates it, a later call with more rows or
 * other chunking may replace it (synchronising `stream` first), and
 * wq_rules_free releases it; the call returns WQ_ERR_OOM if that allocation
 * fails, and WQ_ERR_UNSUPPORTED (from wq_status_check) if the library's compiled chunk
 * lengths are below p + 3 rows.
 * The same row-range, device and stream rules as the forward calls apply;
 * an empty range, or G and H both NULL, gives grad = 0.
 */
wq_status wq_assemble_adjoint(const wq_rules *rules, const double *const *geom, wq_precision prec, const void *G,
                              const void *H, double *grad, int64_t row_begin, int64_t row_end, void *stream);

/*
 * Batched assembly of many independent 3D patches (each its own mesh,
 * degree, map and coefficient; every row of every patch is assembled as in
 * wq_assemble_mass_stiffness, with the weighted Gaussian rules of Sec. 3).
 * The paper treats one patch; the batch is a throughput form of the same
 * computation.  A plan (wq_batch) holds the patches' work lists, folded
 * tables, converted coefficients and partial-contraction buffers, and a CUDA
 * graph of one batched geometry fold, one batched coefficient check and
 * conversion, and per degree two persistent launches (the partial
 * contractions of that degree's patches, then their rows) whose CTAs take
 * work items from global counters.  Its results are bit-identical to one
 * wq_assemble_mass_stiffness call per patch with the same precision.
 */
typedef struct wq_batch wq_batch;
typedef struct {
  const wq_rules *rules;  /* WQ_RULES_DEVICE, dim 3, current device; patches may share one; must outlive the plan */
  const double *geom[3];  /* device control values of the patch's map (n_a doubles each) */
  const double *coef;     /* device coefficient spline, prod(nel_a + 3) doubles, or NULL (c = 1) */
  void *M, *K;            /* device band outputs for all rows of the patch (double for WQ_FP64 and WQ_DF64,
                             float for WQ_MIXED); both required */
} wq_patch;

/*
 * Creates a plan for `npatch` patches (the array is copied; the buffers it
 * points to are read at every launch, so new input values in the same
 * buffers are picked up).  Allocates the plan's device memory once and
 * captures the graph with the default configuration.  WQ_ERR_ARG for a
 * missing pointer, a 2D or host-only rules object, or another device.
 */
wq_status wq_batch_create(const wq_patch *patches, int npatch, wq_precision prec, wq_batch **out);
/* Enqueues the plan's graph on `stream` (asynchronous). */
wq_status wq_batch_launch(wq_batch *batch, void *stream);
/* Synchronises `stream`, returns and clears the plan's device status (as wq_status_check). */
wq_status wq_batch_status(wq_batch *batch, void *stream);
/*
 * Launch configuration: config[0] = chunk length of the row launch (1..32
 * rows of a line), config[1] = resident CTAs per SM of the persistent
 * partial-contraction launch (1..config[4]), config[2] = resident CTAs per SM
 * of the persistent row launch (1..config[5]), config[3] = schedule of the
 * two degrees' launches (each degree has its own pair of kernels; 0: the
 * degree-2 pair on a second stream beside the degree-3 pair, 1: degree 3
 * then degree 2 on one stream; a batch of one degree ignores it).  The CTA
 * counts are capped per kernel at what it can hold.  get writes config[0..5],
 * config[4] and config[5] being the most CTAs per SM the kernels can hold;
 * set reads config[0..3], synchronises the device, rebuilds the work lists
 * and recaptures the graph.
 */
wq_status wq_batch_get_config(const wq_batch *batch, int *config);
wq_status wq_batch_set_config(wq_batch *batch, const int *config);
/*
 * Autotuner: times every configuration of a fixed candidate set (chunk
 * lengths 32/24/16, the two largest CTA counts of each kernel, both schedules),
 * each `reps` times on `stream` after one warm-up (the plan's outputs are
 * written), keeps the fastest and recaptures the graph.  *best_ms (may be
 * NULL) receives its mean time.  Synchronises the device.
 * Persisted cache: when the environment variable WQ_AUTOTUNE_CACHE names a
 * file, the call first looks up the plan's key there -- the GPU (name,
 * compute capability, SM count), the precision, the kernels' occupancy
 * limits, the degree mix, the row count and a hash of the patches' degrees,
 * element counts and coefficient presence -- and, on a hit whose
 * configuration the plan accepts, applies it and returns its stored time
 * without timing anything.  On a miss it times as above and adds or
 * replaces the entry (the file is a JSON object, one entry per line:
 *   "<key>": {"config": [chunk, u_ctas, ctas, schedule], "ms": t}
 * rewritten through a temporary file and a rename; a failed write is not
 * an error).
 */
wq_status wq_batch_tune(wq_batch *batch, void *stream, int reps, double *best_ms);
/* Synchronises the plan's device and frees the plan. */
void wq_batch_free(wq_batch *batch);
/* One-shot form: create, launch on `stream`, check the status, free. */
wq_status wq_assemble_batch(const wq_patch *patches, int npatch, wq_precision prec, void *stream);

/*
 * Valid (in-range column) band entries of rows [row_begin, row_end): the
 * number of CSR entries of that row range.  Host only; -1 on a bad argument.
 */
int64_t wq_band_nnz_rows(const wq_rules *rules, int64_t row_begin, int64_t row_end);

/*
 * Converts band rows [row_begin, row_end) (the layout written by the
 * assembly calls, band = device array of (row_end - row_begin) rows, double
 * for WQ_FP64 and WQ_DF64, float for WQ_MIXED) to CSR on the device:
 *   rowptr  device, row_end - row_begin + 1 int64, rowptr[0] = 0;
 *   col     device, wq_band_nnz_rows(...) int32 global column indices,
 *           increasing within each row;
 *   val     device, as many values of the band's type.
 * Only the entries whose column lies inside the mesh are kept (the band's
 * zeros there are structural, Fig. 1's sparsity pattern).  WQ_ERR_UNSUPPORTED
 * when the mesh has more than 2^31-1 rows (int32 columns).
 */
wq_status wq_band_to_csr(const wq_rules *rules, wq_precision prec, const void *band, int64_t row_begin,
                         int64_t row_end, int64_t *rowptr, int32_t *col, void *val, void *stream);

/*
 * Synchronises `stream`, then returns and clears the device-detected status
 * of the assembly calls made with `rules` since the previous check:
 * WQ_ERR_GEOMETRY if some J_aa <= 0 (or det J <= 0 for wq_assemble_general),
 * WQ_ERR_NONFINITE if some input was NaN or Inf, WQ_ERR_UNSUPPORTED if a
 * kernel met a size it cannot hold (it then writes nothing; not expected for
 * any mesh the rules object accepts), WQ_ERR_CHECK if a range check of a
 * checked build failed, WQ_ERR_CUDA if a kernel failed, else WQ_OK.
 */
wq_status wq_status_check(const wq_rules *rules, void *stream);

/*
 * Assembly that allocates no device memory.  The paper has no counterpart:
 * this is a deployment variant of wq_assemble_mass_stiffness for callers that
 * cannot call cudaMalloc -- a host application whose device memory all
 * belongs to its own pool or arena, or that may not allocate once it is
 * running -- so they cannot hold the device tables a WQ_RULES_DEVICE rules
 * object owns.  Instead, the 1D row tables, the folded geometry tables, the
 * line lists and the status word live in one fixed 8 MiB array in device
 * memory, declared in the library; every GPU that loads the library holds
 * that array until the process exits.
 *
 *   rules        host tables from wq_rules_build (WQ_RULES_HOST_ONLY suffices;
 *                device tables, if any, are not used);
 *   geom, coef   as for wq_assemble_mass_stiffness (device, caller-owned);
 *   M, K         device band outputs as there; either may be NULL to skip
 *                that matrix, not both (unless the range is empty);
 *   check_status 0: return once the work is enqueued on `stream`;
 *                non-zero: synchronise `stream` and return the
 *                device-detected status of this call (WQ_ERR_GEOMETRY,
 *                WQ_ERR_NONFINITE) as wq_status_check would.
 *
 * Returns WQ_ERR_UNSUPPORTED, before touching the GPU, when the mesh's tables
 * do not fit the 8 MiB array (about 1000 elements per direction in 3D; the
 * line lists grow with nel_2 * nel_3).  The call makes no cudaMalloc,
 * cudaFree or other allocating call; it copies the host tables into the
 * array with cudaMemcpyAsync on `stream` every time.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current.
 * All calls on a device share the one array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 */
wq_status wq_assemble_noalloc(const wq_rules *rules, const double *const *geom, const double *coef,
                              wq_precision prec, void *M, void *K, int64_t row_begin, int64_t row_end, void *stream,
                              int check_status);

#ifdef __cplusplus
}
#endif

#endif /* WQ_H */
