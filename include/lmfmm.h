/*
 * lmfmm -- GPU fast multipole method for the interface-induced reaction field
 * of the electric dyadic Green's function of Maxwell's equations in a
 * horizontally layered medium (Yuan, Wang, Zhang, Cai, "Fast Multipole method
 * for Maxwell's equations in layered media", arXiv 2507.18491).
 *
 * Plain C ABI: no C++ or framework types cross it.  Complex numbers are
 * interleaved (re, im) pairs: of double (LMFMM_C128) everywhere, and of float
 * (LMFMM_C64) where a dtype argument allows it.  Every function returns an lmfmm_status
 * (0 = success, negative = error) unless stated otherwise; on error,
 * lmfmm_last_error() returns a one-line description for that context.
 *
 * Physical conventions (Section 3.1): omega = 1 and mu_l = 1 in every layer,
 * so eps_l = k_l^2; layers are numbered 0..L from top to bottom; interface
 * d_l separates layers l and l+1 and d_0 > d_1 > ... > d_{L-1}; every layer
 * wavenumber has Im k_l >= 0.
 *
 * What a matvec computes (eq. layeredmediafields with eq. allcomponents,
 * reaction part, summed over the first Green's-function slot as the paper
 * does):
 *     Phi(r_i) = sum_j sum_{(l,l',*,star)} G^{*star}_{l l'}(r_j, r_i) J_j,
 * over every point j (self term j = i included) and every reaction component
 * whose source layer l holds r_j and whose target layer l' holds r_i.
 *
 * Ownership: the caller owns every buffer it passes; the library owns the
 * tree, the translation tables and its work arrays (device memory it
 * allocates in lmfmm_build and frees in lmfmm_destroy).  Calls on one context
 * are stream-ordered on the stream passed in (NULL = the legacy default
 * stream) and a context must not be used from two host threads at once.
 */
#ifndef LMFMM_H
#define LMFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LMFMM_OK = 0,
    LMFMM_ERR_ARG = -1,          /* invalid argument (NaN, point on an interface, Im k < 0,
                                    non-decreasing interfaces, p out of range, NULL) */
    LMFMM_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    LMFMM_ERR_OOM = -3,          /* device allocation failed */
    LMFMM_ERR_STATE = -4,        /* calls made in the wrong order */
    LMFMM_ERR_QUAD = -5,         /* a bounded quadrature hit its node cap (quad_node_cap) */
    LMFMM_ERR_UNSUPPORTED = -6,  /* request outside what this build implements */
    LMFMM_ERR_TIMEOUT = -7,      /* a bounded device wait of the tensor-core pipeline gave up:
                                    the result of the checked calls is invalid */
    LMFMM_ERR_INTERNAL = -8      /* a consistency check of the library's own setup structures
                                    failed (lmfmm_plan_check) */
} lmfmm_status;

typedef struct lmfmm_ctx lmfmm_ctx;

typedef struct {
    double re, im;
} lmfmm_c128;

enum { LMFMM_FP64 = 0, LMFMM_MIXED = 1 };

/* element type of caller buffers of currents and fields */
enum { LMFMM_C128 = 0, LMFMM_C64 = 1 };

/* parts of the dyadic Green's function a matvec applies (eq. layeredmediafields):
 * the interface-induced reaction field, the free-space part Phi^f of sources in
 * the target's own layer (self term excluded), or both */
enum { LMFMM_REACTION = 0, LMFMM_FREE = 1, LMFMM_TOTAL = 2 };

typedef struct {
    int p;             /* truncation order of the expansions, 1..16 (P = (p+1)^2 coefficients) */
    int depth;         /* octree leaf level (root = 0); < 0 selects it from leaf_cap */
    int leaf_cap;      /* target points per leaf when depth < 0 */
    double theta;      /* admissibility: box pair is far if r_s + r_t <= theta * |c_s - c_t|
                          (centres mapped to images / effective locations) */
    double eta;        /* ... and its vertical transmission distance is >= eta * |c_s - c_t| */
    double quad_tol;   /* relative cut-off of the k_rho tails (>= 1e-16) */
    int precision;     /* LMFMM_FP64 or LMFMM_MIXED (FP32 translation arithmetic) */
    int tensor_cores;  /* mixed form only: products on the tcgen05 tensor cores with FP32-level
                          accuracy.  1: M2L on the persistent kernel (three-piece bf16 split,
                          pre-tiled table image) for p <= 12, else the streamed-operand kernel
                          (three-term TF32 split, p <= 15); 2: the streamed-operand kernel;
                          3: as 1, and M2M / L2L on the persistent kernel too (inputs taken from
                          the highest degree down; four-layer N = 2^20, p = 12: 7.3e-7 against
                          the direct sum, 6.4e-7 with 1); 0: FP32 SIMT pipes.  Beyond p = 15 the
                          SIMT kernel runs.  Ignored by the FP64 form. */
    int quad_node_cap; /* largest k_rho node count of one Sommerfeld integral (an M2L table
                          or a near box pair); beyond it lmfmm_build returns LMFMM_ERR_QUAD
                          (table: checked on the host before any launch; near pair: the
                          device loop is clamped and flags it).  Default 2^20. */
    int components;    /* LMFMM_REACTION (default), LMFMM_FREE or LMFMM_TOTAL.  The free-space
                          part (Section 2) is an FMM of its own over each layer's tree: the
                          same P2M / M2M / L2L / L2P, M2L tables from the addition theorem
                          with the Hessian folded in (host-built, run by the same M2L
                          kernels) and a direct near field in FP64 */
} lmfmm_params;

typedef struct {
    int64_t n_points;
    int n_layers;
    int n_components;      /* active reaction components (l, l', *, star) */
    int depth;
    int64_t n_boxes;       /* non-empty boxes, all layers and levels */
    int64_t n_m2l_pairs;   /* far box pairs, summed over components */
    int64_t n_geometries;  /* distinct (level, rho, z_s, z_t) M2L tables */
    int64_t n_near_pairs;  /* near box pairs */
    int64_t n_near_point_pairs;
    int64_t n_quad_nodes;  /* k_rho nodes summed over all tabulated geometries */
    double bytes_tables;   /* device bytes held by M2L tables (or their tiled tensor-core image) */
    double ms_setup;       /* wall time of the last lmfmm_build */
    double ms_stage[8];    /* last matvec: P2M, M2M, M2L, L2L, L2P, S2T, permute, total */
    int64_t m2l_columns;   /* helical columns pushed through M2L tables per matvec */
    int m2l_kernel;        /* M2L product of the built form: 0 FP64 SIMT, 1 FP32 SIMT,
                              2 tcgen05 streamed-operand kernel, 3 tcgen05 persistent kernel */
    int launches;          /* kernels launched by the last matvec */
    int64_t n_geometries_same_layer;  /* of n_geometries: components with l = l' (their tables
                                         depend on z_s - z_t only and are shared by every
                                         pair of equal (level, rho, z_s - z_t)) */
    double ms_tabulate;    /* last build: M2L tabulation (node factors, Chebyshev integrals,
                              assembly), device time */
    double tab_flops;      /* ... its arithmetic: 8 real flops per complex multiply-add of the
                              Chebyshev integrals (80 (tau, tau', table) combinations x (p+2)
                              degrees x (2p+3) Bessel orders per node) and of the assembly
                              (5 P^2 (p+2) per geometry) */
    int adjoint_transposed; /* 1: lmfmm_matvec_adjoint applies the transposed operators (FP64
                               form, mixed form with tensor_cores = 0); 0: the reciprocity
                               identity with the forward kernels (tensor-core forms) */
    int64_t n_free_geometries;        /* free-space M2L tables (of n_geometries) */
    int64_t n_free_near_point_pairs;  /* free-space near-field point pairs */
} lmfmm_stats;

/* Fill *prm with defaults (p = 8, depth from leaf_cap = 64, theta = 0.55,
 * eta = 0.1, quad_tol = 1e-15, FP64, tensor_cores = 1, quad_node_cap = 2^20,
 * components = LMFMM_REACTION). */
lmfmm_status lmfmm_default_params(lmfmm_params *prm);

/* Create a context on CUDA device `device`.  *out receives the handle. */
lmfmm_status lmfmm_create(lmfmm_ctx **out, const lmfmm_params *prm, int device);

/* Layered medium (Section 3.1): L interfaces d[0..L) (host, strictly
 * decreasing), L+1 layer wavenumbers k[0..L] (host, Im k >= 0, k != 0).
 * L may be 0 (homogeneous space: no reaction field). */
lmfmm_status lmfmm_set_layers(lmfmm_ctx *ctx, int L, const double *d, const lmfmm_c128 *k);

/* N points xyz[N][3] (host, row-major doubles).  A point closer than 1e-12
 * (relative to the domain size) to an interface is ERR_ARG.  Invalidates
 * any previous build. */
lmfmm_status lmfmm_set_points(lmfmm_ctx *ctx, int64_t N, const double *xyz);

/* The same with xyz[N][3] in DEVICE memory, read in order on `stream`; the
 * tree is built on the host, so the call copies the points back and returns
 * after the copy (the caller may free or overwrite xyz afterwards). */
lmfmm_status lmfmm_set_points_device(lmfmm_ctx *ctx, int64_t N, const double *xyz, void *stream);

/* Setup: per-layer octrees, dual-tree traversal of every reaction component
 * into far (M2L) and near (direct) box pairs, deduplication of M2L
 * geometries, device tabulation of the M2L Sommerfeld integrals (Section 3.4)
 * and of the near-field integrals, translation matrices.  Synchronous. */
lmfmm_status lmfmm_build(lmfmm_ctx *ctx, void *stream);

/* Phi = A J with A the reaction-field operator above.  J[N][3] and Phi[N][3]
 * are DEVICE pointers in the caller's point order, both of element type
 * `dtype` (LMFMM_C128 or LMFMM_C64; complex64 currents are widened exactly and
 * the complex128 sum is rounded once into a complex64 Phi); Phi is
 * overwritten.  Asynchronous on `stream`: argument and state errors are
 * returned at once, while a device-side failure (LMFMM_ERR_TIMEOUT) is
 * reported by lmfmm_check after the call has run. */
lmfmm_status lmfmm_matvec(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi, void *stream);

/* Same operator with HOST buffers J[N][3], Phi[N][3] of element type dtype:
 * copies in, applies, copies out; returns after Phi is written, with the
 * device status checked (lmfmm_check).  Pinned host memory is faster. */
lmfmm_status lmfmm_matvec_host(lmfmm_ctx *ctx, const void *J, int dtype, void *Phi, void *stream);

/* out = A^T y, A the FMM operator as built (device buffers of element type
 * dtype): every stage of the matvec replaced by its exact transpose, in
 * reverse order -- the transposed helical maps, L2P^T (point values summed
 * against the L2P functions into the leaf local expansions), L2L^T and M2M^T
 * (transposed translation matrices, up and down the tree), M2L^T (transposed
 * tables with the same per-pair factors), P2M^T (multipole expansions
 * evaluated with the P2M functions) and the transposed near field.  So
 * <x, A^T y> = <A x, y> holds to rounding, whatever the truncation.  FP64 form
 * and mixed form with tensor_cores = 0 (LMFMM_ERR_UNSUPPORTED otherwise: the
 * tensor-core forms keep their tables only as the tiled image).  By
 * reciprocity (G(r,r') = G(r',r)^T, invoked by the paper for the first-slot
 * sum) A^T approximates A itself.  Asynchronous like lmfmm_matvec. */
lmfmm_status lmfmm_matvec_transpose(lmfmm_ctx *ctx, const void *y, int dtype, void *out, void *stream);

/* Phi = A^H y (device buffers of element type dtype): conj(A^T conj(y)) with
 * the transposed operator above where the form has it (stats
 * adjoint_transposed = 1); in the tensor-core forms the reciprocity identity
 * A^H y = conj(A conj(y)) with the forward kernels.  Asynchronous. */
lmfmm_status lmfmm_matvec_adjoint(lmfmm_ctx *ctx, const void *y, int dtype, void *Phi,
                                  void *stream);

/* Vector-Jacobian product of the FP64 form for a real objective L of the field
 * E = A(r) J: given J[N][3] and g = dL/dconj(E) [N][3] (DEVICE, element type
 * dtype), writes gJ = A^H g (dtype; may be NULL) and gxyz[N][3] (DEVICE
 * doubles, caller order; may be NULL) with
 *     gxyz_j = Re sum_i conj(g_i) . dE_i/dr_j,
 * the derivative of the operator with the tree, lists and quadrature rules
 * held fixed: the local expansions at r_j (target role, L2P's functions
 * differentiated), the multipole functions at r_j contracted with the
 * transposed pass's expansions (source role), and the near-field integrals
 * differentiated in rho, phi and the image heights.  Runs a forward pass and
 * the transposed pass, checkpointing the forward local expansions and
 * helical charges in between.  The first call allocates the checkpoints and
 * 20 derivative integrals per near point pair.  LMFMM_ERR_UNSUPPORTED outside
 * the FP64 form.  Asynchronous on stream. */
lmfmm_status lmfmm_gradient(lmfmm_ctx *ctx, const void *J, const void *g, int dtype, void *gJ, double *gxyz,
                            void *stream);

/* Waits for `stream` and reads the context's device status word, which every
 * matvec clears (stream-ordered) before its first kernel.  Returns LMFMM_OK,
 * LMFMM_ERR_TIMEOUT if a bounded wait inside a tensor-core kernel of the
 * matvecs since then gave up (that result is incomplete), or LMFMM_ERR_CUDA. */
lmfmm_status lmfmm_check(lmfmm_ctx *ctx, void *stream);

/* Test hook for the error path above: ORs `bits` into the device status word
 * from the host (synchronous), as a tensor-core wait that gives up would.
 * Bit 4 is the only meaning defined today.  Requires lmfmm_build. */
lmfmm_status lmfmm_test_set_status(lmfmm_ctx *ctx, int bits);

/* Direct evaluation of the same operator over ALL point pairs with the
 * device near-field kernel (Sommerfeld integral per pair, Section 3.5);
 * O(N^2), intended for N up to a few thousand.  Device buffers. */
lmfmm_status lmfmm_direct(lmfmm_ctx *ctx, const lmfmm_c128 *J, lmfmm_c128 *Phi, void *stream);

/* The same all-pairs direct evaluation as lmfmm_direct, for callers that
 * cannot allocate device memory during the call: programs whose device
 * memory is wholly reserved by another allocator (a framework's caching
 * pool, say), or that must not stall or fail on an allocation mid-run.  The
 * paper has no counterpart; this is a property of the library, not of the
 * method.  It calls no cudaMalloc, cudaFree or allocating library routine:
 * its scratch (leaf-pair list + 5 complex Sommerfeld coefficients per point
 * pair) is one file-scope device array of 32 MiB, and the pair list is
 * built in a fixed host array of 65536 records.  Requires lmfmm_build (the
 * context's own buffers, allocated there, are reused).  Returns
 * LMFMM_ERR_ARG, with the byte count in the message, when
 * (leaf pairs * 48 bytes, rounded up to 256) + (point pairs * 80 bytes)
 * exceeds 32 MiB -- about N^2 <= 4e5 point pairs over all components.
 * The array is shared by every call on a device and keeps the last call's
 * contents; the call zero-fills what must start at zero.  The array, the
 * host pair list and the per-device address cache are process-wide, so the
 * call holds a process-wide lock from the pair list to its final wait: calls
 * from several host threads (any contexts, any devices) run one at a time
 * and never overlap on the GPU.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  J, Phi: DEVICE [N][3] complex, caller's
 * point order; synchronous (returns after Phi is written). */
lmfmm_status lmfmm_direct_noalloc(lmfmm_ctx *ctx, const lmfmm_c128 *J, lmfmm_c128 *Phi,
                                  void *stream);

/* Density functions phi^{*star}_{l lp}, psi^{*star}_{l lp} (eq. threedensity)
 * at n nodes krho[n] (DEVICE, complex).  out[n][8] (DEVICE): phi for
 * (up,up),(up,dn),(dn,up),(dn,dn) then psi in the same order, where the first
 * arrow is the direction at the target (first slot, layer l) and the second
 * at the source (second slot, layer lp).  Requires lmfmm_set_layers. */
lmfmm_status lmfmm_densities(lmfmm_ctx *ctx, int l, int lp, int64_t n, const lmfmm_c128 *krho,
                             lmfmm_c128 *out, void *stream);

/* Sommerfeld integrals I-hat (eq. onedimensionintegral) of one M2L geometry
 * for component (l, lp, tgt_up, src_up), via the Chebyshev expansion of
 * Section 3.4 (eqs. legendre_Q_v/w, chebyshev_integral_I).  out (DEVICE)
 * [5][P][P] complex, P = (p+1)^2, tables in the order (sigma1,kappa 0),
 * (sigma5,0), (sigma2,1), (sigma4,1), (sigma3,2); row = target index
 * nu^2+nu+mu, column = source index n^2+n+m; Bessel order m - mu + kappa.
 * (rho, zs, zt): horizontal distance and heights of the source and target
 * centres after mapping to image / effective coordinates. */
lmfmm_status lmfmm_m2l_table(lmfmm_ctx *ctx, int l, int lp, int tgt_up, int src_up, double rho,
                             double zs, double zt, lmfmm_c128 *out, void *stream);

/* Host-only (no device, no context): the M2M and L2L matrices of the
 * regular expansions used by the reaction-field FMM (Section 3.3 notes that
 * the layered ME/LE bases are those of the Helmholtz equation, so M2M/L2L
 * are eqs. maxwell_M2M_freespace / maxwell_L2L_freespace).  For wavenumber k
 * and shift t = child centre - parent centre (t[3], host):
 *   m2m[P][P]: parent ME = m2m * child ME,   l2l[P][P]: child LE = l2l * parent LE,
 * row-major, index n^2+n+m, P = (p+1)^2, 1 <= p <= 16; host arrays owned by
 * the caller.  Built from the addition theorem with exact Gaunt
 * coefficients, so small entries are accurate relative to their own size. */
lmfmm_status lmfmm_translation_matrix(int p, lmfmm_c128 k, const double *t, lmfmm_c128 *m2m,
                                      lmfmm_c128 *l2l);

/* Host-only (no device, no context): the free-space M2L of the FMM's free
 * part (Section 2, eq. maxwell_M2L_freespace with the Hessian of eq.
 * GEandGH) between a source box centre c_s and a target centre c_t with
 * c_s - c_t = (rho, 0, dz), wavenumber k, as the library stores it: tables
 * [5][P][P] in the five-table form of lmfmm_m2l_table (same order, row =
 * target index, column = source index, P = (p+1)^2), so that the M2L kernels
 * apply it with the reaction tables' per-pair factors; blocks [3][3][P][P]
 * (optional, NULL to skip) the full operator from the helical multipole
 * expansions (a, b, c) to the helical local expansions of the field at this
 * azimuth.  Caller-owned host arrays; 1 <= p <= 16. */
lmfmm_status lmfmm_free_m2l_table(int p, lmfmm_c128 k, double rho, double dz, lmfmm_c128 *tables,
                                   lmfmm_c128 *blocks);

/* Host-only (no device, no context): the Chebyshev form of the normalised
 * associated Legendre functions that the M2L tabulation uses (Appendix B).
 * For 0 <= m <= n <= p (1 <= p <= 16), with t = n (n + 1) / 2 + m and
 * K = (p + 1) / 2, B[t][0 .. K] (caller-owned, (p+1)(p+2)/2 x (K+1) doubles)
 * holds the coefficients with
 *     P^_n^m(cos b) = tau_nm(b) sum_j B[t][j] T_j(cos 2b),
 *     tau_nm = 1 (n, m even), 1 / cos b (n odd, m even), sin b (n, m odd),
 *              sin b / cos b (n even, m odd),
 * an identity of polynomials in (cos b, sin b), so it holds for the complex
 * angles of the Sommerfeld integrals (cos b = k_z / k, sin b = k_rho / k);
 * entries past a function's degree are 0. */
lmfmm_status lmfmm_legendre_chebyshev(int p, double *B);

/* Host-only: the product tensor of eqs. legendre_Q_v / legendre_Q_w that the
 * tabulation contracts with the Chebyshev integrals (Section 3.4 with Appendix
 * A's C^{ab} re-expansion of T_j(a x + b)): for source and target wavenumbers
 * k, kp and every source index s = (n', m') and target index t = (nu, mu)
 * (triangle indices as above, T = (p+1)(p+2)/2), G[s][t][0 .. p+1]
 * (caller-owned, T x T x (p+2) complex) satisfies
 *     f_s(b) f_t(b') = sum_l G[s][t][l] T_l(cos 2 b0),
 * f = P^ / tau of lmfmm_legendre_chebyshev, cos 2b = 1 - 2 k_rho^2 / k^2,
 * cos 2b' = 1 - 2 k_rho^2 / kp^2, b0 the angle of the smaller of |k|, |kp|. */
lmfmm_status lmfmm_legendre_product(int p, lmfmm_c128 k, lmfmm_c128 kp, lmfmm_c128 *G);

/* Counts of the built context and the timings of its last build and matvec
 * (fields above; the stage times are CUDA-event intervals on the matvec's
 * stream, filled in once its last event has completed, else those of the
 * previous matvec).  No synchronisation.  *out is caller-owned. */
lmfmm_status lmfmm_get_stats(const lmfmm_ctx *ctx, lmfmm_stats *out);

/* ------------------------------------------------------------- plan check
 * The setup structures of lmfmm_build, built and checked on the host alone (no
 * device is touched, no context is kept): the per-layer octrees over the sorted
 * points, the dual traversal of every reaction component (l, l', *, star) into
 * far box pairs and near leaf pairs (Sections 3.3 and 3.4.1; admissibility as in
 * lmfmm_params), the distinct M2L geometries and their pair lists, the
 * free-space lists when params->components asks for them (Section 2), the
 * M2M / L2L translation groups and the 64-column M2L work items of the
 * persistent tensor-core kernel.  Checks:
 *   tree       every layer's points are partitioned by the boxes of each level,
 *              children partition their parent, every point lies in its leaf's
 *              cell, box radii bound their points;
 *   coverage   every (component, source leaf, target leaf) triple is reached by
 *              exactly one far pair of some ancestor pair or one near pair (the
 *              FMM's split of the double sum), likewise every same-layer leaf
 *              pair of the free-space part;
 *   geometry   every far pair meets the admissibility test and has the
 *              horizontal distance, mapped heights (or, within a layer, height
 *              offset) and direction of its geometry's table;
 *   indices    every box, pair, geometry, coefficient offset and work-item range
 *              a kernel reads is in bounds, and pair ranges tile their arrays.
 * Arguments as lmfmm_create / lmfmm_set_layers / lmfmm_set_points (host xyz,
 * [N][3] double); flags: 0, or the test hooks below, which remove one pair
 * after the build so that a caller can see the check report it.  Coverage is
 * checked per component and target leaf, as a tiling of the source leaves by
 * the intervals its ancestors' far pairs and its near pairs reach, while a
 * component has at most 2^25 such intervals (larger ones are counted in
 * n_components_unchecked).  Host memory ~24 bytes per interval.  Returns
 * LMFMM_OK when every check holds, LMFMM_ERR_INTERNAL when one fails (the
 * count and the first failure are in *out), or the argument error of the
 * corresponding context call (message in out->message). */
enum { LMFMM_PLAN_DROP_FAR_PAIR = 1, LMFMM_PLAN_DROP_NEAR_PAIR = 2 };

typedef struct {
    int depth;                      /* leaf level */
    int n_components;               /* reaction components */
    int n_free_components;          /* free-space pseudo-components (one per layer with points) */
    int n_components_unchecked;     /* components whose coverage was too large to check */
    int64_t n_boxes;
    int64_t n_leaves[9];            /* per layer (at most 9 layers) */
    int64_t n_far_pairs, n_geometries, n_near_pairs, n_near_point_pairs;
    int64_t n_free_far_pairs, n_free_geometries, n_free_near_pairs, n_free_near_point_pairs;
    int64_t n_translation_pairs;    /* (child, parent) pairs of the M2M / L2L groups */
    int64_t n_work_items, n_columns;   /* M2L work items (<= 64 helical columns) and columns */
    int64_t n_leaf_pairs_checked;   /* (component, source leaf, target leaf) triples covered */
    int64_t n_violations;           /* failed checks (0: consistent) */
    double root_center[3], root_half;  /* root cell; leaves have side 2 root_half / 2^depth */
    int64_t n_geometries_level[21]; /* reaction M2L tables per tree level, all components */
    int64_t max_geometries_component_level;  /* most tables of one (component, level) */
    char message[256];              /* first failure or argument error, else empty */
} lmfmm_plan_info;

lmfmm_status lmfmm_plan_check(const lmfmm_params *prm, int L, const double *d, const lmfmm_c128 *k,
                              int64_t N, const double *xyz, int flags, lmfmm_plan_info *out);

/* Leaf-level tuner (host only): for every depth dmin..dmax (<= 10) the setup
 * structures are built as above and the matvec time predicted from their counts,
 *   t = u0 (M2L work items) + u1 (near point pairs, both parts) + u2 (M2M / L2L
 *       child-parent pairs) + u3 N   [ns],
 * with unit_ns = {u0, u1, u2, u3}, or NULL for costs measured on GB300 with the
 * mixed form and the tensor-core M2L / M2M / L2L at p = 12 (about 80, 0.27, 14.7
 * and 1.1 ns), scaled to other p by (P / 169)^2 (u0, u2) and P / 169 (u3).  The
 * accuracy is set by theta and p, not by the depth.  predicted_ms[dmax - dmin + 1]
 * receives the predictions, *best the depth of the smallest.  Errors as
 * lmfmm_plan_check (LMFMM_ERR_ARG also for a bad depth range or NULL outputs). */
lmfmm_status lmfmm_plan_depth(const lmfmm_params *prm, int L, const double *d, const lmfmm_c128 *k,
                              int64_t N, const double *xyz, int dmin, int dmax, const double *unit_ns,
                              int *best, double *predicted_ms);

/* ------------------------------------------------------------- batches
 * Many layered problems (own media, points, sizes; one device, one p, one
 * precision) applied together.  lmfmm_batch_matvec records every problem's
 * upward pass, one merged persistent M2L launch over all problems' work items
 * (when every problem runs the persistent tensor-core M2L, i.e. the mixed
 * form with tensor_cores 1 or 3 and p <= 12; otherwise each problem's own
 * M2L), and every downward pass into a CUDA graph on its first call, and
 * replays that graph while the caller's pointers stay the same (new
 * pointers: a new capture).  The contexts stay owned by the caller and must
 * outlive the batch; a batch must not be used from two host threads at once. */
typedef struct lmfmm_batch lmfmm_batch;

lmfmm_status lmfmm_batch_create(lmfmm_batch **out, lmfmm_ctx *const *ctxs, int n);

/* Phi[i] = A_i J[i] for every problem i: J, Phi host arrays of n DEVICE
 * pointers, each [N_i][3] of element type dtype.  Asynchronous on stream (the
 * graph runs there); device-side failures via lmfmm_batch_check. */
lmfmm_status lmfmm_batch_matvec(lmfmm_batch *b, const void *const *J, void *const *Phi, int dtype,
                                void *stream);

/* Autotuner of the merged M2L's work tiles: times the persistent launch
 * (device events, best of three after a warm run, on zeroed expansions) with
 * the work items cut to 64 or 32 helical columns (one MMA tile of 128 real
 * rows, or half of it) and ordered problem by problem or round robin, and
 * keeps the fastest (lmfmm_batch_info).  Synchronous.  LMFMM_ERR_UNSUPPORTED
 * when the batch has no merged M2L. */
lmfmm_status lmfmm_batch_tune(lmfmm_batch *b, void *stream);

/* Waits for stream; LMFMM_ERR_TIMEOUT if a bounded tensor-core wait of the
 * batch's launches gave up. */
lmfmm_status lmfmm_batch_check(lmfmm_batch *b, void *stream);

/* merged: 1 if the M2L runs as one launch; nwork: its work items; variant:
 * the tuned tiling (bit 0 round robin, bit 1 32-column items); ms_variant[4]:
 * the tuner's timings (0 before lmfmm_batch_tune).  Any pointer may be NULL. */
lmfmm_status lmfmm_batch_info(const lmfmm_batch *b, int *merged, int64_t *nwork, int *variant,
                              double *ms_variant);

const char *lmfmm_batch_last_error(const lmfmm_batch *b);
void lmfmm_batch_destroy(lmfmm_batch *b);

/* Never NULL; valid until the next call on ctx.  ctx may be NULL (creation
 * errors). */
const char *lmfmm_last_error(const lmfmm_ctx *ctx);

void lmfmm_destroy(lmfmm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* LMFMM_H */
