/*
 * lhv.h -- C ABI of the GB300 Lamb-Helmholtz vortex FMM (liblhv.so).
 *
 * The library evaluates, for N vortex elements with positions x_i and strength
 * vectors w_i, the velocity and the vortex-stretching term of Eq. s1.1 of
 * Gumerov & Duraiswami, "Efficient FMM accelerated vortex methods in three
 * dimensions via the Lamb-Helmholtz decomposition":
 *
 *   v_i = sum_{j != i} K(|x_i - x_j|; a) w_j x (x_i - x_j) / |x_i - x_j|^3   (Eqs. 1, 2)
 *   s_i = (w_i . grad) v |_{x_i}                                           (Eq. s1.1)
 *
 * with the Gaussian core K of Eq. vem1 (K = 1 when a = 0), and advances
 * (x_i, w_i) by dx/dt = v, dw/dt = s with classical RK4 (Sec. 5.3).  The far
 * field is carried by the two harmonic potentials phi and chi of Eq. 4, with the
 * conversion operators of Eqs. drt10/drt11 applied after every translation
 * (Sec. 4); the near field (colleague leaves) is summed directly.
 *
 * Conventions shared by every entry point:
 *  - Element buffers are caller-owned DEVICE memory (unless the name ends in
 *    _host), contiguous [n][4]: float4 for the FP32 entry points, double[4]
 *    (32-byte aligned) for the _f64 ones.  Lanes 0..2 hold (x, y, z) or
 *    (w_x, w_y, w_z); lane 3 is ignored on input and written 0 on output.
 *  - Outputs are in the caller's element order.
 *  - All work is enqueued on the stream given to lhv_create, in stream order.
 *    Calls that build a tree read a few sizes back to the host (two short
 *    synchronisations of that stream per tree build), except the steps replayed
 *    from a captured graph (lhv_set_graph: one synchronisation per RK4 step).
 *  - Every call returns a status code (LHV_OK = 0, negative on error); no C++
 *    exception crosses the ABI.  After an error the outputs are unspecified and
 *    the context stays usable; lhv_last_error() describes the last error.
 *  - The context owns every internal buffer (tree, expansions, operator tables,
 *    RK4 stages); it is freed by lhv_destroy.
 */
#ifndef LHV_H
#define LHV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define LHV_OK            0
#define LHV_EINVAL       -1  /* bad argument: null/misaligned pointer, n < 0, p out of range, a < 0 */
#define LHV_ENOMEM       -2  /* device allocation failed */
#define LHV_ECUDA        -3  /* a CUDA runtime call or kernel launch failed */
#define LHV_ETIMEOUT     -4  /* a device-side bounded wait gave up */
#define LHV_ENONFINITE   -5  /* NaN or Inf in the positions or strengths */
#define LHV_EUNSUPPORTED -6  /* valid request this library does not implement */
#define LHV_ETOOBIG      -7  /* input larger than the fixed scratch of a no-allocation entry point */

/* ---- arithmetic of the evaluation (lhv_config.precision) --------------- */
#define LHV_FP32 0  /* all kernels in FP32 (CUDA cores); operator tables built in FP64, stored FP32 */
#define LHV_FP64 1  /* all kernels in FP64 (use the _f64 entry points) */
#define LHV_TF32X3 2 /* mixed precision: as LHV_FP32, but the M2L products run on the tensor cores
                        in TF32 with split operands (hi.hi + hi.lo + lo.hi, FP32 accumulation)
                        where p is a multiple of 4; other p and the other maps run as in
                        LHV_FP32 */

/* ---- which parts of Eq. fmm1 to evaluate (lhv_config.terms) ------------ */
#define LHV_TERMS_NEAR 1  /* sparse part only: direct sum over colleague leaves */
#define LHV_TERMS_FAR  2  /* dense part only: P2M, M2M, M2L, L2L, L2P */
#define LHV_TERMS_ALL  3

typedef struct lhv_ctx lhv_ctx;

typedef struct {
    int    p;          /* truncation number: terms n = 0 .. p-1 (Sec. 5.1); 1 <= p <= 24 */
    int    leaf_max;   /* leaf bound: leaf level = shallowest level with <= leaf_max
                          elements per box, capped by the core rule below; >= 1 */
    double core_a;     /* Gaussian core a of Eq. vem1; 0 selects the singular Eq. 1 */
    double eps;        /* target accuracy in (0, 1): leaf boxes are kept no smaller
                          than r_K = x_K a with 1 - K(x_K a; a) = eps/10, so far pairs
                          see K = 1 to eps/10 (Eq. 2) */
    int    precision;  /* LHV_FP32, LHV_FP64 or LHV_TF32X3 */
    int    terms;      /* LHV_TERMS_* (0 means LHV_TERMS_ALL) */
    int    max_level;  /* cap on the leaf level, 0 = none (21, the key depth) */
} lhv_config;

#define LHV_MAX_LEVELS 22
#define LHV_NUM_STAGES 12
/* stage indices of lhv_stats.stage_ms */
#define LHV_STAGE_TREE   0  /* Morton keys, sort, boxes, lists */
#define LHV_STAGE_P2M    1  /* Sec. 4.3 */
#define LHV_STAGE_M2M    2  /* Sec. 4.4, S conversion Eq. drt11 */
#define LHV_STAGE_M2L    3  /* Sec. 4.4, R conversion Eq. drt10 */
#define LHV_STAGE_L2L    4  /* Sec. 4.4, R conversion Eq. drt10 */
#define LHV_STAGE_L2P    5  /* Sec. 4.5 */
#define LHV_STAGE_P2P    6  /* Eq. fmm1 sparse part, Eqs. 2 and vem1 */
#define LHV_STAGE_RK4    7  /* Sec. 5.3 RK4 combine */
#define LHV_STAGE_OPS    8  /* FP64 operator build (once per context) */
#define LHV_STAGE_COPY   9  /* host <-> device copies of the _host entry points */
#define LHV_STAGE_M2L_PRODUCTS 10  /* the operator products of M2L alone (inside LHV_STAGE_M2L) */
#define LHV_STAGE_SELECT 11  /* learned form: features, network and choice (tree excluded) */

typedef struct {
    int     leaf_level;                      /* L of the last tree */
    int     nbox[LHV_MAX_LEVELS];            /* occupied boxes per level of the last tree */
    int64_t n;                               /* elements of the last tree */
    int64_t p2p_pairs;                       /* ordered (target, source) pairs, j != i, of the
                                                last near-field evaluation */
    int64_t m2l_pairs;                       /* (target, source) box pairs of the last M2L */
    double  stage_ms[LHV_NUM_STAGES];        /* summed device time per stage since the last
                                                reset (only while timing is enabled) */
    int64_t stage_launches[LHV_NUM_STAGES];  /* timed stage executions since the last reset */
    int64_t kernel_launches;                 /* kernels launched since the last reset */
    int     level_p[LHV_MAX_LEVELS];         /* truncation number of each level's expansions in
                                                the last evaluation with a far field (0: none) */
    int     selector_leaf_max;               /* leaf cap of the last selection (0: none yet) */
    int64_t selector_selections;             /* selections since lhv_set_selector */
    int64_t selector_checks;                 /* sampled direct-sum checks since then */
    int64_t selector_fallbacks;              /* checks that failed (fixed p used instead) */
    double  selector_err_v, selector_err_s;  /* relative L2 error of v and s on the sample at the
                                                last check (-1: none) */
    int     tuned_p2p_targets_per_thread;    /* launch shapes in use (lhv_autotune) */
    int     tuned_p2p_sources_per_stage;
    int     tuned_m2l_pairs_per_chunk;       /* 0: the default (128 on the tensor cores, else
                                                the largest CUDA-core chunk that fits) */
    int     tuned_m2l_tensor_cores;          /* 1 when M2L runs on the tensor cores */
    double  tune_ms[12];                     /* stage times of the candidates, in the order
                                                P2P 1/2/4 targets per thread at 128 sources per
                                                stage, the same at 256, then M2L: (TF32x3 only:
                                                tensor cores 128, 64 pairs,) CUDA cores 64, 32,
                                                16 pairs */
    int64_t graph_captures;                  /* steps captured as a CUDA graph (lhv_set_graph) */
    int64_t graph_replays;                   /* steps run as one replay of the captured graph */
    int64_t graph_fallbacks;                 /* steps whose tree failed the captured layout's guard
                                                and ran uncaptured */
    int64_t graph_kernels;                   /* kernels in the captured graph */
} lhv_stats;

/* Create a context for one configuration on one CUDA stream (a cudaStream_t,
 * NULL = the legacy default stream) of the current device.  *out receives the
 * handle.  Returns LHV_EINVAL for a null cfg/out or out-of-range fields. */
int lhv_create(const lhv_config* cfg, void* cuda_stream, lhv_ctx** out);

/* Free every buffer the context owns.  NULL is accepted. */
void lhv_destroy(lhv_ctx* ctx);

/* Static text for a status code. */
const char* lhv_status_string(int status);

/* Text of the last error of this context (empty when none). */
const char* lhv_last_error(lhv_ctx* ctx);

/* Build the octree of n FP32 positions (device [n][4]): cube, Morton keys,
 * stable sort, boxes per level, colleague lists (Sec. 4, "Create data
 * structure").  The cube: origin at the per-axis minimum; side the smallest
 * r_q 2^k >= the largest extent, r_q the core radius r_K (where the Gaussian core
 * of Eq. vem1 is 1 to eps/10) rounded up to an 8-bit mantissa, so that one level's
 * box side lies in [r_K, 1.008 r_K); without a core (core_a = 0) the smallest
 * power of two >= the largest extent.  Leaf level: the shallowest with at most
 * leaf_max elements per box, no deeper than the deepest whose box side is >= r_K.
 * Evaluation calls rebuild it themselves; this entry point exists to time or
 * inspect the tree alone. */
int lhv_build_tree(lhv_ctx* ctx, int64_t n, const float* x4);

/* v and s (Eq. s1.1) of n elements: x4, w4 in, v4, s4 out (device [n][4], FP32
 * context).  Builds the tree of x4 first.  n = 0 is a no-op. */
int lhv_evaluate_velocity_stretching(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4,
                                     float* v4, float* s4);

/* One classical RK4 step of Eq. s1.1 in place on x4 and w4 (device [n][4],
 * FP32 context); four evaluations, each with its own tree (Sec. 5.3). */
int lhv_step(lhv_ctx* ctx, int64_t n, float* x4, float* w4, double dt);

/* lhv_step on HOST buffers (pageable or pinned [n][4] FP32): copies in, steps,
 * copies back, all on the context stream; returns when the results are in
 * x4_host and w4_host. */
int lhv_step_host(lhv_ctx* ctx, int64_t n, float* x4_host, float* w4_host, double dt);

/* Batched form: nsys independent systems in one call.  System k owns the
 * elements [offsets[k], offsets[k+1]) of x4/w4/v4/s4 (offsets: HOST int64
 * [nsys+1], offsets[0] = 0, non-decreasing; 1 <= nsys <= 4096).  Systems do not
 * interact; each gets its own cube and octree, all trees are built, translated
 * and summed by the same launches.  One leaf level serves the whole batch: the
 * deepest any system needs, capped by the core rule of the smallest cube.  With a
 * core (core_a > 0) every system's cube takes the largest side of the batch (its
 * origin stays its own), so that the capped leaf level gives every system leaves
 * of side r_q (see lhv_build_tree).
 * Morton keys keep the system id in their top bits and use
 * floor((63 - ceil(log2 nsys)) / 3) bits per axis.  FP32 / TF32X3 contexts. */
int lhv_evaluate_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, const float* x4, const float* w4,
                         float* v4, float* s4);
int lhv_step_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, float* x4, float* w4, double dt);

/* FP64 twins (FP64 context; element buffers are double[n][4], 32-byte aligned). */
int lhv_evaluate_velocity_stretching_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* w4,
                                         double* v4, double* s4);
int lhv_step_f64(lhv_ctx* ctx, int64_t n, double* x4, double* w4, double dt);

/* The paper's reference case (Sec. 5.2, Tables 1-2): the scalar harmonic FMM for the
 * potential and its gradient of n monopoles of strength q_j,
 *   phi(x_i) = sum_{j != i} q_j / |x_i - x_j|,  grad phi(x_i) = -sum_{j != i} q_j (x_i - x_j) / |x_i - x_j|^3
 * (no 1/(4 pi), like Eq. 1; distinct elements at one point contribute nothing), on the same
 * octree, lists and kernels as the vortex evaluation with one potential: P2M by the Green's
 * expansion (Eq. rsbf5), M2M / M2L / L2L by the translation block of each fused operator
 * (no conversion: there is no chi), L2P of phi and grad phi, and the direct sum over the
 * colleague leaves.  It is what the ratio T(v, s) / T(phi, grad phi) of Sec. 5.2 is
 * measured against.  x4: device [n][4] positions (lane 3 ignored); q: device [n] charges
 * (float / double, not checked for NaN/Inf); pg4: device [n][4] output in the caller's
 * order, lanes (d phi/dx, d phi/dy, d phi/dz, phi).  Uses lhv_config.p at every level
 * (per-level p and the selector do not apply), leaf_max, max_level, terms and, for
 * LHV_TF32X3, the tensor-core M2L products where p^2 is a multiple of 16.  The context
 * must have core_a = 0 (the singular Laplace kernel of the reference case):
 * LHV_EUNSUPPORTED otherwise.  LHV_EINVAL for null or misaligned pointers, n < 0, or a
 * precision that does not match the entry point (FP32 / TF32X3 contexts for the float
 * form, FP64 for _f64). */
int lhv_evaluate_potential_gradient(lhv_ctx* ctx, int64_t n, const float* x4, const float* q, float* pg4);
int lhv_evaluate_potential_gradient_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* q, double* pg4);

/* Vortex filaments (Sec. 5.3, App. B): v at the nodes of nfil polylines.  Filament f owns
 * the nodes [offsets[f], offsets[f+1]) of x4 (offsets: HOST int64 [nfil+1], offsets[0] = 0,
 * non-decreasing); segment k runs from node k to node k + 1, or from the last node back to
 * the first when closed[f] != 0 (closed: HOST int32 [nfil]), with constant circulation
 * gamma[k] (device [n], the segment that starts at node k; unused for the last node of an
 * open filament).  Each node receives, from every segment that does not start or end at
 * it, the closed form of Eq. dis2,
 *   v = gamma / (4 pi) (r1 x r2) / (r1 r2 + r1 . r2) (1/r1 + 1/r2),  rj = node - end j,
 * summed by the FMM: the octree of the nodes, each segment in the leaf of its first node;
 * far field from its S-expansion by Gauss-Legendre quadrature with [(p - 1)/2] + 1 points
 * (Eqs. vf5-vf7: Eq. eve4 with (gamma / 8 pi) l in place of w), the near field in closed
 * form over the segments of the colleague leaves (a node on a segment's line gets 0 from
 * it).  Segments should be short against the leaf side.  v4: device [n][4] output in the
 * caller's order (lane 3 written 0).  Needs core_a = 0, the two-potential form and the
 * selector off (LHV_EUNSUPPORTED otherwise); LHV_EINVAL for bad offsets or pointers, or a
 * precision that does not match the entry point. */
int lhv_evaluate_filaments(lhv_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closed, const float* x4,
                           const float* gamma, float* v4);
int lhv_evaluate_filaments_f64(lhv_ctx* ctx, int nfil, const int64_t* offsets, const int32_t* closed,
                               const double* x4, const double* gamma, double* v4);

/* The exact sum the FMM approximates, at m sampled targets: v and s of Eq.
 * s1.1 with the kernel of Eqs. 2/vem1 (the context's core_a) summed over every
 * element j != idx[k] (excluded by index), in FP64 arithmetic.  This is the
 * measure of the FMM error on a sample of targets (Sec. 5.1 uses 1000 points).
 * x4, w4: the n elements (device [n][4], FP32 for lhv_direct_sampled, FP64 for
 * the _f64 twin on an FP64 context); idx: device int32 [m] caller indices;
 * v4, s4: device double [m][4] (32-byte aligned) outputs.  With core_a = 0
 * coincident distinct elements contribute nothing (the singular kernel has no
 * value there).  Synchronous on the context stream; O(m n) work.  Returns
 * LHV_EINVAL for an index outside [0, n). */
int lhv_direct_sampled(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, int m, const int32_t* idx,
                       double* v4, double* s4);
int lhv_direct_sampled_f64(lhv_ctx* ctx, int64_t n, const double* x4, const double* w4, int m, const int32_t* idx,
                           double* v4, double* s4);

/* Autotuner (launch shapes, not in the paper): runs the evaluation of the given
 * elements once per candidate and keeps, for this context, the fastest P2P tile
 * shape (1, 2 or 4 targets per thread: FP32 warp tiles of 32, 64 or 128 targets,
 * FP64 blocks of 128, 64 or 32 threads over tiles of 128 targets; times 128 or 256
 * sources staged in shared memory per step) and the
 * fastest M2L grouping (box pairs of one offset per GEMM chunk: 64, 32 or 16 on
 * the CUDA cores; under TF32X3 also the tensor-core kernel with 128 or 64 pairs
 * per chunk), chosen by CUDA-event stage times (best of 3 after a warm-up).  v4
 * and s4 receive the last evaluation.  The batched twin tunes on a batch
 * (offsets as for lhv_evaluate_batched).  Results do not depend on the choice
 * beyond rounding. */
int lhv_autotune(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, float* v4, float* s4);
int lhv_autotune_batched(lhv_ctx* ctx, int nsys, const int64_t* offsets, const float* x4, const float* w4,
                         float* v4, float* s4);
/* Set the launch shapes directly: P2P targets per thread (1, 2, 4) and sources per
 * stage (128, 256), M2L pairs per CUDA-core chunk (16, 32, 64, or 0 for the
 * default), M2L on the tensor cores (1) or not (0; only TF32X3 contexts use
 * them).  LHV_EINVAL otherwise. */
int lhv_set_launch_shape(lhv_ctx* ctx, int p2p_targets_per_thread, int p2p_sources_per_stage,
                         int m2l_pairs_per_chunk, int m2l_tensor_cores);

/* Truncation number per octree level (variable truncation, which the paper
 * mentions but does not use, Sec. 5).  p[l] for the levels l < nlevels (host
 * array; 1 <= p[l] <= 24, or 0 for lhv_config.p); levels >= nlevels, and every
 * level after nlevels = 0, use lhv_config.p.  The expansions of level l (S at the
 * leaves and above, R from level 2 down) then have p[l] terms: P2M and L2P use
 * p[L], M2L at level l maps p[l] -> p[l], M2M level l+1 -> l maps p[l+1] ->
 * p[l] and L2L level l -> l+1 maps p[l] -> p[l+1] (each result truncated to
 * its level's p before the conversion of Eqs. drt10/drt11).  Tables of other
 * (p_out, p_in) pairs are built in FP64 on first use and kept by the context.
 * Takes effect at the next evaluation.  LHV_EINVAL for values out of range. */
int lhv_set_level_p(lhv_ctx* ctx, const int* p, int nlevels);

/* Whole RK4 step as one CUDA graph (enable = 1; 0 switches it off and frees the graph).
 * Applies to lhv_step, lhv_step_batched and lhv_step_host on FP32 / TF32X3 contexts with
 * one truncation number at every level and the selector off (other steps run as usual).
 * The first step after enabling (and after any change of n, the system offsets, the
 * x4 / w4 pointers, dt, p, precision, form or launch shapes) runs uncaptured, then in the
 * captured layout, and is captured for the next calls; each later step is one
 * cudaGraphLaunch on the context stream followed by one 4-byte read and a stream
 * synchronisation.  The captured layout: the leaf level of the capture's first tree is
 * kept for every tree of the replayed steps, box arrays sit at per-level capacities
 * min(n, nsys 8^l) so that no launch needs a size read back, every kernel takes the box
 * counts from device memory, the sort orders the full keys, and a device guard keeps the
 * step from writing x4, w4 when a tree fails it (a NaN/Inf input, or a cube whose core
 * rule no longer allows the kept level); such a step is redone uncaptured (its
 * LHV_ENONFINITE reported as usual) and the graph is captured again at the next step.
 * Results equal the uncaptured step's to rounding (the same kernels; atomic additions in
 * another order).  Stage timing (lhv_set_timing) records nothing inside captured steps;
 * lhv_get_stats reads the box counts from the device after them; lhv_export refuses the
 * box and expansion arrays of a tree built by a captured step (LHV_EUNSUPPORTED).
 * Needs a context created on a stream other than the legacy default stream
 * (LHV_EUNSUPPORTED otherwise); LHV_EINVAL for enable other than 0 or 1. */
int lhv_set_graph(lhv_ctx* ctx, int enable);

/* Representation of the far field (Sec. 4.2).  LHV_FORM_PHI_CHI (the default): the two
 * real potentials phi and chi, p^2 reals each, translated by the fused real tables
 * [[T, C12 T], [0, C22 T]] (translation and conversion, zero block skipped).
 * LHV_FORM_PSI: one complex harmonic function Psi = phi + i chi (Eq. chf1), stored as
 * 2 p^2 reals (Re / Im of Psi_n^m for m >= 0, then of Psi_n^{-m}; Im Psi_n^0 in place of
 * the m = 0 entry of the second half), translated by one dense real table per offset or
 * octant, M F M^-1, with M the change of layout (Psi_n^m = phi_n^m + i chi_n^m, Psi_n^{-m}
 * = (-1)^m (conj phi_n^m + i conj chi_n^m)) and F the fused table: one complex translation
 * of Psi plus the conversions of Eqs. drt10/drt11 on the potentials split from it.  P2M
 * produces (phi, chi) by Eq. eve4 and converts the leaf rows to Psi; L2P splits the leaf
 * locals back.  In the scaled basis (see lhv_export) Psi combines the scaled phi and
 * chi coefficients, i.e. Psi = phi + i h chi at box side h.  The complex form needs one
 * truncation number at every level (LHV_EUNSUPPORTED at evaluation under
 * lhv_set_level_p values or the selector); lhv_export then returns Psi rows for
 * LHV_EXPORT_MULTIPOLE / LHV_EXPORT_LOCAL.
 * LHV_FORM_RCR: the two potentials as in LHV_FORM_PHI_CHI, with every M2L translation
 * done by rotation - coaxial translation - back rotation (Sec. 4.4, Fig. 1b): the
 * coefficients of each potential are rotated degree by degree into the frame whose z
 * axis is t, translated along z by |t|, converted by the coaxial form of Eq. drt10
 * (Eq. rcr1) and rotated back; O(p^3) per translation on the CUDA cores instead of the
 * O(p^4) fused table.  M2M and L2L keep the fused tables (one per box).  Tables are
 * built in FP64 at the first evaluation (synchronous).  FP32 only, one truncation
 * number p <= 20 at every level: LHV_EUNSUPPORTED at evaluation otherwise (FP64
 * precision, lhv_set_level_p values, the selector, p > 20).  The results equal those of
 * the other forms up to rounding.  LHV_EINVAL for another value. */
#define LHV_FORM_PHI_CHI 0
#define LHV_FORM_PSI     1
#define LHV_FORM_RCR     2
int lhv_set_form(lhv_ctx* ctx, int form);

/* Statistics of the last tree/evaluation and the accumulated stage timings. */
int lhv_get_stats(lhv_ctx* ctx, lhv_stats* out);

/* Enable (1) or disable (0) per-stage CUDA-event timing on the context stream. */
int lhv_set_timing(lhv_ctx* ctx, int enable);

/* Zero the accumulated stage timings and the launch counter. */
int lhv_reset_stats(lhv_ctx* ctx);

/* Copy an internal array of the last tree/evaluation into a caller DEVICE
 * buffer of capacity_bytes (stream-ordered).  *bytes_out receives the size of
 * the array (also when dst is NULL, to query it).  `level` selects the octree
 * level where the array is per level.  Returns LHV_EINVAL if the array does
 * not exist or does not fit.  Arrays:                                         */
#define LHV_EXPORT_KEYS        1  /* uint64[n] Morton keys in the tree's order: sorted (stable)
                                     for a context's first tree and whenever the context has no
                                     core radius and no level cap; otherwise sorted by their
                                     prefix down to five levels below the deepest level that the
                                     core rule and the level cap allowed in the previous tree,
                                     equal prefixes in input order (the boxes of every level the
                                     tree uses are the same) */
#define LHV_EXPORT_PERM        2  /* int32[n] sorted position -> caller index */
#define LHV_EXPORT_BOX_KEYS    3  /* uint64[nbox(level)] key prefixes of the level's boxes */
#define LHV_EXPORT_BOX_RANGE   4  /* int32[nbox(level)][2] sorted element range [begin, end) */
#define LHV_EXPORT_COLLEAGUES  5  /* int32[nbox(level)][27] colleague box index or -1,
                                     offset (dx,dy,dz) at ((dx+1)*3+(dy+1))*3+(dz+1) */
#define LHV_EXPORT_MULTIPOLE   6  /* real[nbox(level)][2][p*p] scaled S coefficients (phi, chi),
                                     p = the level's truncation number (lhv_stats.level_p) */
#define LHV_EXPORT_LOCAL       7  /* real[nbox(level)][2][p*p] scaled R coefficients (phi, chi) */
#define LHV_EXPORT_CUBE        8  /* double[4]: x0, y0, z0 of the (first system's) cube and its side */
/* Scaled real coefficient layout (both potentials, box side h at that level):
 * real index n*n for Re c_n^0, n*n + 2m - 1 / n*n + 2m for Re / Im c_n^m (m >= 1);
 * S coefficients are stored as  c_n^m nu_n^m / h^(n+1) (phi) and c_n^m nu_n^m / h^n (chi),
 * R coefficients as             c_n^m h^n / nu_n^m (phi)    and c_n^m h^(n+1) / nu_n^m (chi),
 * nu_n^m = sqrt((n-|m|)! (n+|m|)!), c_n^m the coefficients of Eq. rsbf6. */
int lhv_export(lhv_ctx* ctx, int what, int level, void* dst, int64_t capacity_bytes, int64_t* bytes_out);

/* ---- no-allocation entry point ------------------------------------------
 * The paper has no counterpart to this call: it is an engineering variant of the
 * first step of lhv_build_tree (cube, Morton keys and stable sort of one system,
 * Sec. 4, "Create data structure") for callers that must not allocate device
 * memory, because cudaFree synchronises the whole device (cudaMalloc may too)
 * and both can fail or stall when a caching allocator already holds the device
 * memory: a real-time loop that shares the GPU with other streams, a host
 * callback, or an application that owns a fixed memory budget.  It allocates nothing (no
 * cudaMalloc/cudaFree, no allocating library routine): every temporary lives in
 * one file-scope device array of fixed size (about 12.3 MiB, present once the
 * library's module is loaded on a device), whose address the first call on each
 * device looks up (cudaGetSymbolAddress).  That first call also loads the
 * library's kernels on the device; make it before any stream capture begins and
 * outside any region that cannot tolerate that one-time setup.
 *
 * Inputs: n <= LHV_NOALLOC_MAX_N positions x4 (device float [n][4], 16-byte
 * aligned) and optional strengths w4 (same layout, or NULL; only checked for
 * NaN/Inf).  Outputs (caller-owned device memory, also used as one side of the
 * sort's ping-pong): keys (uint64 [n]) the sorted Morton keys and perm (int32
 * [n]) sorted position -> caller index, identical to LHV_EXPORT_KEYS and
 * LHV_EXPORT_PERM after lhv_build_tree of the same positions in a new context or
 * one without core radius and level cap (21 bits per axis, stable order of
 * equal keys).  Work is enqueued on cuda_stream (a cudaStream_t,
 * NULL = legacy default stream); the call returns after that stream has
 * finished it (one device-to-host read of the non-finite flag).  The only
 * scratch state that must start at zero (the non-finite flag) is cleared by the
 * call's first kernel.  Returns LHV_ETOOBIG for n > LHV_NOALLOC_MAX_N,
 * LHV_EINVAL for n < 0, null or misaligned pointers, LHV_ENONFINITE for NaN/Inf,
 * LHV_ECUDA if a CUDA call failed, LHV_OK for n = 0 (nothing done).  A CUDA
 * error already pending on the calling thread when the call starts (from the
 * caller's earlier work) makes it return LHV_ECUDA before launching anything,
 * with that error left in place for the caller to read; any CUDA error after
 * that point is this call's own.
 * Calls that overlap in time on one device (from several host threads, or on
 * several streams without ordering between them) share the one scratch array
 * and race: the caller serialises them. */
#define LHV_NOALLOC_MAX_N (1 << 20)
int lhv_morton_sort_noalloc(int64_t n, const float* x4, const float* w4, uint64_t* keys, int32_t* perm,
                            void* cuda_stream);

/* ---- selector network of the learned form -------------------------------
 * The paper uses one truncation number for the whole tree (Sec. 5 names a
 * variable truncation number among the optimisations it left out).  The learned
 * form picks one per level with a multilayer perceptron over 12 features of the
 * level: h1 = relu(W1 x + b1) (12 -> 64), h2 = relu(W2 h1 + b2) (64 -> 64),
 * h3 = relu(W3 h2 + b3) (64 -> 64), z = W4 h3 + b4 (64 -> 21); z[0..16] score
 * p = 4 .. 20, z[17..20] score the leaf caps 16, 32, 64, 128.  Weights are
 * bfloat16 (W: uint16 bit patterns, W1, W2, W3, W4 row-major (out x in) one
 * after the other, LHV_MLP_NW values), biases FP32 (b1..b4, LHV_MLP_NB values);
 * all arithmetic and accumulation is FP32.  These three calls are stateless:
 * every pointer is caller-owned DEVICE memory, work is enqueued on cuda_stream
 * (a cudaStream_t, NULL = legacy default stream); LHV_EINVAL for rows < 0 or a
 * null pointer, LHV_ECUDA if a launch failed. */
#define LHV_MLP_IN     12
#define LHV_MLP_HIDDEN 64
#define LHV_MLP_OUT    21
#define LHV_MLP_NP     17
#define LHV_MLP_NW     10304
#define LHV_MLP_NB     213
/* Z [rows][21] = logits of the feature rows X [rows][12]. */
int lhv_mlp_forward(int rows, const float* X, const uint16_t* W, const float* b, float* Z, void* cuda_stream);
/* Loss of a batch and its gradient: yp [rows] (p label 0..16, or -1 for none),
 * yl [rows] (leaf label 0..3 or -1); loss = mean cross-entropy over the rows
 * with a p label + mean cross-entropy over the rows with a leaf label.  gW
 * (float [LHV_MLP_NW]), gb (float [LHV_MLP_NB]) and loss (float [1]) are
 * overwritten with the gradient with respect to the weights (taken at their
 * bfloat16 values) and biases; work: device int [2] scratch. */
int lhv_mlp_loss_grad(int rows, const float* X, const int32_t* yp, const int32_t* yl, const uint16_t* W,
                      const float* b, float* gW, float* gb, float* loss, int32_t* work, void* cuda_stream);
/* One Adam step (Kingma & Ba 2015; beta1 0.9, beta2 0.999, eps 1e-8) of step
 * number t >= 1 on the FP32 master weights W32 and biases b with moments
 * (mW, vW), (mb, vb); W receives the bfloat16 rounding (to nearest even) of W32. */
int lhv_mlp_adam(float* W32, uint16_t* W, const float* gW, float* mW, float* vW, float* b, const float* gb,
                 float* mb, float* vb, int t, float lr, void* cuda_stream);

/* Learned form on a context (FP32 or TF32X3; single-system entry points).
 * lhv_set_selector copies the network (HOST arrays W: LHV_MLP_NW bfloat16
 * bit patterns, b: LHV_MLP_NB floats; W = NULL switches the form off) and sets
 * the target eps: the relative L2 error of v against the direct sum on a sample
 * of check_samples elements (Sec. 5.1 uses 1000).  Then every
 * lhv_evaluate_velocity_stretching, and every lhv_step / lhv_step_host from its
 * initial state, first builds the tree at lhv_config.leaf_max, scores levels
 * 2..L with the network, and evaluates with p[l] = 4 + argmax of the p scores of
 * level l and leaf cap = {16, 32, 64, 128}[argmax of the leaf scores of level L]
 * (an lhv_step keeps that choice for its four stages).  The first selection
 * and every check_every-th after it (0: never) is checked: the FP64 direct sums
 * of lhv_direct_sampled at the sample against the evaluation; if the error of v
 * exceeds eps the evaluation is redone with lhv_config.p at every level and
 * lhv_config.leaf_max (the fixed-p fallback).  lhv_get_stats reports the
 * choices, checks and fallbacks.  While the form is on, the selector replaces
 * any lhv_set_level_p values.  LHV_EINVAL for eps outside (0, 1), check_samples
 * < 1, or an FP64 context. */
int lhv_set_selector(lhv_ctx* ctx, const uint16_t* W, const float* b, double eps, int check_every,
                     int check_samples);
/* The network's input for n FP32 elements: builds their tree (x4, w4 device
 * [n][4]) and writes one row of LHV_MLP_IN features per level l = 2..L (row
 * l - 2) into X (device float [capacity_rows][LHV_MLP_IN]); *rows_out = L - 1
 * (0 when the tree has no far field; X may be NULL to query it).  eps is the
 * target that enters the features.  Feature list (each scaled to about
 * [-1, 1]): l/10, (L-l)/10, log2(boxes at l)/20, log2(boxes(l)/boxes(l-1))/3,
 * log2(n/boxes at l)/20, -log10(eps)/10, log2(a/h_l)/10 (-3 when a = 0),
 * mean interaction-list size/189, mean colleague count/27,
 * log10(sum_b |sum_{j in b} w_j| / sum_j |w_j|)/3, log2(n)/24, and 0 / 0.5
 * for FP32 / TF32X3. */
int lhv_selector_features(lhv_ctx* ctx, int64_t n, const float* x4, const float* w4, double eps, float* X,
                          int capacity_rows, int* rows_out);

/* Diagnostic: D = X B^T on the TF32 tensor-core path of this library, one CTA,
 * operands rounded to TF32 (no splitting).  X: device float [128][K], B: device
 * float [N][K], D: device float [128][N]; 16 <= N <= 256 with N % 16 == 0 and
 * K % 32 == 0.  Synchronous on the legacy default stream.  Returns LHV_EINVAL
 * for other sizes, LHV_ETIMEOUT if the tensor-core work never signalled
 * completion (the kernel then stops by itself). */
int lhv_tc_selftest(const float* X, const float* B, float* D, int N, int K);

/* ---- throughput probes (the roofline denominators; not in the paper) ------
 * Measures, at the GPU's current clocks (nothing is set or locked), the rate of
 * one pipe with a register- or shared-memory-resident loop and no global traffic:
 *   LHV_PEAK_FFMA      FP32 fused multiply-add, scalar fmaf (flop/s, 2 per lane-op)
 *   LHV_PEAK_FFMA2     FP32 fused multiply-add, packed FP32x2 (flop/s, 4 per lane-op;
 *                      the form of the near-field pair loop)
 *   LHV_PEAK_MUFU      SFU reciprocal square root rsqrt.approx (operations/s)
 *   LHV_PEAK_TF32_MMA  tcgen05.mma kind::tf32, 128 x 256 x 8 (flop/s, dense)
 *   LHV_PEAK_BF16_MMA  tcgen05.mma kind::f16 with BF16 operands, 128 x 256 x 16 (flop/s)
 * The FP32 and SFU probes run every SM at full occupancy, `iters` loop trips of 128
 * operations per thread; the tensor probes 2 CTAs per SM, `iters` MMAs each.  One
 * warm-up launch, then `reps` timed launches (CUDA events on cuda_stream, a
 * cudaStream_t, NULL = legacy default stream); *rate_out receives the rate of the
 * median launch and *ms_out (may be NULL) its duration.  Synchronous; allocates
 * and frees a few bytes of device memory.  LHV_EINVAL for an unknown probe or
 * iters, reps < 1; LHV_ECUDA if a CUDA error is pending on entry or a launch
 * fails; LHV_ETIMEOUT if the tensor-core completion wait gave up (bounded). */
#define LHV_PEAK_FFMA     1
#define LHV_PEAK_FFMA2    2
#define LHV_PEAK_MUFU     3
#define LHV_PEAK_TF32_MMA 4
#define LHV_PEAK_BF16_MMA 5
int lhv_peak_probe(int what, int iters, int reps, void* cuda_stream, double* rate_out, double* ms_out);

#ifdef __cplusplus
}
#endif

#endif /* LHV_H */
