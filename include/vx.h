/*
 * vx.h -- C ABI of libvx: CSF-amortized interval subdivision on one GB300 (sm_103a).
 *
 * The method is that of G. Moroz, "Sparse Tensors and Subdivision Methods for Finding the
 * Zero Set of Polynomial Equations" (arXiv 2406.09857): the boxes of one subdivision level
 * are stored as a Compressed Sparse Fiber tree (Sec. 2.1), the polynomials are evaluated
 * on all of them at once by partial evaluation along the tree (Algorithm 2 built on the
 * Horner scheme of Algorithm 1, cost given by Theorem 1), boxes whose interval value does
 * not contain 0 are dropped (criterion C0, Sec. 3.2), and the survivors are bisected 2^k
 * ways into the next level (Algorithm 3).
 *
 * Conventions shared by every call:
 *   - Every call returns VX_OK (0) or a negative VX_E* code and never aborts, throws or traps;
 *     vx_last_error() then holds a message for the calling thread.
 *   - Pointers prefixed h_ are host memory, d_ device memory of the current CUDA device.
 *     Caller-owned buffers stay owned by the caller; objects returned through an out-pointer
 *     (vx_system, vx_csf, vx_result) are owned by the caller and released by the matching
 *     *_free call, which frees their device memory in the order of the stream they were made
 *     on (that stream must still exist then).  `stream` is a cudaStream_t (NULL = the legacy
 *     default stream); all device work of a call is ordered on it, and device outputs are
 *     valid once it has reached them.
 *   - Variable x_1 is at the root of the CSF and x_k at the leaves; children are in
 *     ascending label order, so leaves are in lexicographic order of their index tuples.
 *   - A grid level l splits axis i of the domain [lo_i, hi_i] into 2^l boxes
 *     [lo_i + t w_i, lo_i + (t+1) w_i], w_i = (hi_i - lo_i) / 2^l.  The domain must be finite
 *     with lo_i < hi_i and every grid point of the level must be exactly representable in
 *     binary64 (dyadic domains such as [-1,1]^k or [0,1]^k); otherwise VX_EINVAL.
 *   - 1 <= k <= VX_KMAX variables, 1 <= npoly <= VX_MAXPOLY polynomials, levels 0..VX_MAXLEVEL.
 */
#ifndef VX_H
#define VX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VX_OK 0
#define VX_EINVAL (-1)    /* an argument is out of range or malformed */
#define VX_ENOMEM (-2)    /* a host or device allocation failed */
#define VX_ECAPACITY (-3) /* a caller-provided buffer or a fixed limit is too small */
#define VX_EOVERFLOW (-4) /* a node count would not fit the 32-bit node indices */
#define VX_ETIMEOUT (-5)  /* a bounded device wait gave up */
#define VX_ECUDA (-6)     /* a CUDA runtime call failed */

#define VX_KMAX 6
#define VX_MAXPOLY 16
#define VX_MAXLEVEL 24

/* Arithmetic of a level evaluation. */
#define VX_FP64 0        /* binary64 intervals [lo, hi]: lower ends rounded down, upper up */
#define VX_FP32_MIDRAD 1 /* binary32 midpoint-radius <m, r> with the rounding error of every
                          * step bounded a priori and added to r, so the enclosure contains
                          * the exact range (and the VX_FP64 enclosure) */
#define VX_FP32 2        /* binary32 approximations of the VX_FP64 interval ends (rounded to
                          * nearest) carrying an a-priori bound on their distance to them: a box
                          * whose binary32 value is farther than that bound from deciding C0
                          * either way is decided in binary32, the others are re-evaluated in
                          * VX_FP64, so every keep decision equals the VX_FP64 one (the values
                          * d_lo/d_hi it returns are within that bound of the VX_FP64 ones) */

/* Relation of a polynomial F of a system of equations and inequalities (Sec. 4: the input is
 * equations and inequalities).  C0 drops a box when F's enclosure on it proves the relation
 * false on the whole box: VX_EQ when 0 is outside, VX_LE when lo > 0, VX_GE when hi < 0,
 * VX_LT when lo >= 0, VX_GT when hi <= 0. */
#define VX_EQ 0 /* F = 0 */
#define VX_LE 1 /* F <= 0 */
#define VX_GE 2 /* F >= 0 */
#define VX_LT 3 /* F < 0 */
#define VX_GT 4 /* F > 0 */

/* Inclusion criteria C1 for one equation (Sec. 3.2, "Inclusion Criterion"); a box C1
 * certifies holds a zero of F (F has certified opposite signs at two of its points). */
#define VX_C1_TAYLOR 1 /* the Taylor form of order m >= 2 at the vertices V_max, V_min where its
                        * linear part is largest / smallest (s_i = sign of the midpoint of
                        * G_{e_i}(c), lo >= -hi counting as +): lower bound at V_max > 0 and
                        * upper bound at V_min < 0 */
#define VX_C1_VERTEX 2 /* F at the 2^k vertices (Algorithm 2 on point intervals): one vertex
                        * certified > 0 and another < 0 */

/* One polynomial: nterms monomials coefs[t] * prod_i x_i^exps[t*nvars+i] (Sec. 2.1,
 * "Representing a Multivariate Polynomial").  Host memory, borrowed for the duration of the
 * call.  Exponents >= 0, no monomial twice, coefficients finite. */
typedef struct {
  int32_t nvars;
  int32_t nterms;
  const int32_t *exps; /* [nterms][nvars] */
  const double *coefs; /* [nterms] */
} vx_poly;

typedef struct vx_system vx_system; /* packed polynomials, resident on the device */
typedef struct vx_csf vx_csf;       /* a CSF of box indices of one grid level, on the device */
typedef struct vx_result vx_result; /* the outcome of an enclosure */

/* Options of vx_enclose*: zero-initialise, then set what you need (all-zero = VX_FP64). */
typedef struct {
  int32_t mode;         /* VX_FP64, VX_FP32 or VX_FP32_MIDRAD (for the levels below the last
                         * when fp64_final is set) */
  int32_t fp64_final;   /* VX_FP32_MIDRAD only: evaluate the last level in VX_FP64, which makes
                         * the result exactly the VX_FP64 result (VX_FP32 needs no such step:
                         * its every level is the VX_FP64 level) */
  int32_t fp64_recheck; /* VX_FP32_MIDRAD only: boxes kept by the FP32 test with |m| >= theta*r
                         * for some polynomial are re-evaluated in VX_FP64 at the same level */
  float theta;          /* recheck threshold, 0 < theta <= 1 (0 means 0.5) */
  int32_t timing;       /* nonzero: time every kernel launch with CUDA events (vx_result_timing) */
  int32_t taylor_order; /* 0: C0 on nested interval Horner (Algorithm 2); m >= 1: C0 on the
                         * Taylor form of order m (Def. 3), VX_FP64 or VX_FP32 (certified: the
                         * decisions of VX_FP64); the number of multi-indices |a| <= m
                         * (C(m+k, k)) must not exceed VX_MAXPOLY */
  int32_t c1;           /* 0, VX_C1_TAYLOR (needs taylor_order >= 2) or VX_C1_VERTEX: Algorithm 3
                         * with the inclusion criterion, one equation, VX_FP64 or VX_FP32 (the
                         * same decisions; vertex signs in binary64).  From level
                         * c1_level on (the boxes below the size threshold) the boxes C1
                         * certifies leave the subdivision and are returned with their level
                         * (vx_result_included); the loop ends when no box is left or after
                         * level `depth`, whose remaining boxes are vx_result_boxes */
  int32_t c1_level;
  int32_t small_level_madds; /* VX_FP32 only, 0 = off: a level (of vx_enclose*) whose interval
                              * multiply-adds (Theorem 1's count; times the Taylor form's
                              * derivatives) are fewer than this runs in VX_FP64, which decides
                              * every box as VX_FP32 does and on a level too small to fill the
                              * GPU is faster than binary32 plus its band check */
  int32_t recheck_last; /* VX_FP32 on the interval form (taylor_order 0, c1 0) only: the boxes
                         * inside the error band stay in S at the levels below the last one and
                         * only the last level's are re-decided in binary64.  The final boxes
                         * are still exactly VX_FP64's: C0 on interval Horner is inclusion-
                         * isotone over the exact grids (a box that binary64 drops has every
                         * descendant dropped by binary64 too), so keeping a box that binary64
                         * would drop changes only the counts of the levels in between
                         * (vx_result_stats), never the boxes that the last level keeps */
  int32_t max_level_boxes; /* 0 = 2^31 - 1: the most boxes one tree may hold at a level.  A
                            * level whose kept boxes would give the next level more is run in
                            * ranges of consecutive x_1 slabs, each through the remaining levels
                            * on its own, in x_1 order (a box's descendants stay in its slab and
                            * every box is decided on its own, so the result is the same); the
                            * final boxes are then several trees, joined by vx_result_csf while
                            * they fit one.  VX_EOVERFLOW when one slab alone exceeds it.  Not
                            * with c1 (whose inclusion step keeps levels whole) */
  int32_t first_level; /* 0 = off; on the interval form (taylor_order 0, c1 0): Algorithm 3 starts
                        * from the full grid of level min(first_level, depth) instead of level 0.
                        * The final boxes are the same (C0 on interval Horner is inclusion-isotone
                        * over exact grids, so pruning the coarser levels changes no final box);
                        * the levels before it are not evaluated (zero in vx_result_stats) and the
                        * start level tests its whole grid.  For levels that keep nearly every box,
                        * whose launches cost more than their few boxes */
  int32_t host_codes;  /* nonzero (vx_enclose*): the last level's compaction writes every final
                        * box's grid-index code (vx_result_box_codes' format) straight into pinned
                        * host memory as it places the box, so that the codes cross the host link
                        * while the compaction runs; vx_result_box_codes then returns them without
                        * a copy.  Ignored (the codes are made on the first vx_result_box_codes
                        * call) when the final boxes are several trees (max_level_boxes) */
} vx_opts;

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *vx_last_error(void);

/* Packs the polynomials F_list[0..npoly) (all in the same number of variables k) for the
 * device and uploads them on `stream` (Sec. 2.1: the exponent CSF, laid out fibre-major so
 * that Algorithm 1 runs along contiguous rows).  The system holds device memory until
 * vx_system_free. */
int vx_system_create(const vx_poly *F_list, int32_t npoly, void *stream, vx_system **out);
/* vx_system_create for a system of equations and inequalities with interval coefficients
 * (Sec. 4; coefficients such as sqrt(3) enter as the binary64 interval around them):
 * coefs_hi (nullable; entries nullable) gives per polynomial the upper ends of its
 * coefficients, F_list[f].coefs being the lower ends (lower <= upper, both finite); rel
 * (nullable: all VX_EQ) the relation of each polynomial.  Every path honours both, except
 * the tensor-core dense level (vx_dense_plan_create refuses such systems) and C1 (one
 * equation only). */
int vx_system_create_ex(const vx_poly *F_list, const double *const *coefs_hi,
                        const int32_t *rel, int32_t npoly, void *stream, vx_system **out);
void vx_system_free(vx_system *sys);
/* k and npoly of a system; h_M (nullable) receives [npoly][k+1] the number of coefficients
 * each partial-evaluation stage reads: M_{j} for j = 0..k, with missing suffix monomials below
 * the highest exponent of a fibre counted as zero coefficients (M_k = 1). */
int vx_system_info(const vx_system *sys, int32_t *k, int32_t *npoly, int64_t *h_M);
/* The same counts without a device: packs F_list[0..npoly) on the host only (the checks of
 * vx_system_create: exponents, finite coefficients, no monomial twice) and writes h_M
 * [npoly][k+1] as vx_system_info does.  Touches no GPU. */
int vx_system_measure(const vx_poly *F_list, int32_t npoly, int64_t *h_M);

/* Bytes of device memory the packed system holds (what vx_system_create uploads). */
int vx_system_device_bytes(const vx_system *sys, int64_t *bytes);
/* Bytes vx_system_create copied from the host (the packed binary64 coefficients and the
 * stage tables; the binary32 encodings are made on the device from them). */
int vx_system_upload_bytes(const vx_system *sys, int64_t *bytes);
/* Number of kernels this library has launched in this process so far (all threads). */
int64_t vx_kernel_launches(void);
/* Failure-path hook: how many times a kernel polls for a bulk copy before it gives up, on the
 * current device (a negative value restores the default, 2^22; 0 gives up at once).  A kernel
 * that gives up records it, still waits (with the default bound) for its own copy to land,
 * and returns without results; the call then fails with VX_ETIMEOUT.  Not part of
 * Algorithm 3. */
int vx_set_wait_limit(int64_t polls);

/* The CSF (Sec. 2.1) of n box indices d_tuples[n][k] (device, int32, lexicographically
 * strictly increasing, each coordinate in [0, 2^level)) of grid level `level`.  Depth-j nodes
 * are the distinct length-j prefixes (Remark 1: there are N_j(S) of them).  VX_EINVAL if the
 * tuples are not strictly increasing or out of range (checked on the device). */
int vx_csf_build(int32_t k, int32_t level, const int32_t *d_tuples, int64_t n, void *stream,
                 vx_csf **out);
/* The CSF of every box of grid level `level`: the dense grid X_1 x ... x X_k of Property 1
 * (Sec. 1.1), on which Algorithm 2's stages are the mode-by-mode partial evaluation of the
 * coefficient tensor.  (2^level)^k boxes, at most 2^31 (VX_EOVERFLOW).  Filled directly. */
int vx_csf_full_grid(int32_t k, int32_t level, void *stream, vx_csf **out);
void vx_csf_free(vx_csf *csf);
/* k, level and h_N[k] = N_1..N_k (nodes per depth; N_k = number of boxes). */
int vx_csf_nodes(const vx_csf *csf, int32_t *k, int32_t *level, int64_t *h_N);
/* Copies depth `depth` (1..k) of the tree: d_labels[N_depth] (grid index of each node along
 * x_depth), and for depth < k d_ptr[N_depth + 1] (children of node i are nodes d_ptr[i] ..
 * d_ptr[i+1]-1 of depth+1).  d_ptr may be NULL. */
int vx_csf_export(const vx_csf *csf, int32_t depth, int32_t *d_labels, int32_t *d_ptr,
                  void *stream);
/* Writes the index tuples of the leaves, d_tuples[N_k][k], in leaf (lexicographic) order. */
int vx_csf_tuples(const vx_csf *csf, int32_t *d_tuples, void *stream);

/* Algorithm 2 on every leaf box of `csf` with the C0 test of Sec. 3.2.
 * h_domain[2k]: lo_i, hi_i per axis (host).  mode: VX_FP64 or VX_FP32_MIDRAD.
 * d_keep[N_k] (required): 1 if 0 lies in the interval value of every polynomial, else 0
 * (VX_FP32: the VX_FP64 decision, boxes inside the error band being re-evaluated in binary64).
 * d_lo, d_hi [npoly][N_k] (both NULL or both set): the enclosure of each polynomial on each
 * box (VX_FP32_MIDRAD: m - r rounded down and m + r rounded up, in binary64; VX_FP32: the
 * binary32 bounds).
 * Returns once the evaluation is complete (it synchronises `stream`); VX_ETIMEOUT if a bounded
 * wait inside a kernel gave up (the outputs are then not valid).
 * In VX_FP64 mode every endpoint equals the CPU statement of Algorithms 1-2 with outward
 * rounding (RD of each product and sum for lower ends, RU for upper ends, the product of
 * intervals as the hull of the endpoint products). */
int vx_csf_eval_level(const vx_system *sys, const vx_csf *csf, const double *h_domain,
                      int32_t mode, double *d_lo, double *d_hi, uint8_t *d_keep, void *stream);

/* C0 on the Taylor form of order m >= 1 (Def. 3, Sec. 3.2) instead of nested interval Horner:
 * with c the centre of a box and x - c in [-r, r],
 *   T_m(F, B) = sum_{|a| < m} G_a(c) (x - c)^a + sum_{|a| = m} []G_a(B) (x - c)^a,
 * G_a = (d^a F / dx^a) / a! (interval coefficients: the integer factors times the binary64
 * coefficients rounded both ways), G_a(c) by Algorithm 2 on the centres' point intervals and
 * []G_a(B) on the boxes, (x - c)^a as the exact range of each variable's power, the terms
 * summed in lexicographic order of a with outward rounding; keep = 0 in every polynomial's
 * form.  Binary64 only.  C(m+k, k) must not exceed VX_MAXPOLY.  d_lo/d_hi (nullable,
 * [npoly][N_k] binary64) receive T; d_keep [N_k].  Synchronises `stream`. */
int vx_csf_eval_level_taylor(const vx_system *sys, const vx_csf *csf, const double *h_domain,
                             int32_t order, double *d_lo, double *d_hi, uint8_t *d_keep,
                             void *stream);

/* C0 on the Taylor form of order m >= 1 (as vx_csf_eval_level_taylor) and, when d_inc is
 * non-null (m >= 2, one equation), C1 on it (VX_C1_TAYLOR), in mode VX_FP64 or VX_FP32: the
 * latter evaluates the derivatives in certified binary32, brackets each binary64 value between
 * a narrow and a wide interval and decides as binary64 does wherever both agree, the other
 * boxes by the binary64 form (*n_recheck, nullable, receives how many).  d_keep / d_inc
 * [N_k] device, caller-owned.  Synchronises `stream`. */
int vx_csf_taylor_level(const vx_system *sys, const vx_csf *csf, const double *h_domain,
                        int32_t order, int32_t mode, uint8_t *d_keep, uint8_t *d_inc,
                        int64_t *n_recheck, void *stream);

/* The inclusion criterion C1 (kind VX_C1_TAYLOR with `order` >= 2, or VX_C1_VERTEX; see
 * their definitions) of the system's one polynomial on every leaf box of the level:
 * d_inc[N_k] (device, caller-owned) = 1 where certified.  Binary64.  Synchronises `stream`. */
int vx_csf_c1(const vx_system *sys, const vx_csf *csf, const double *h_domain, int32_t kind,
              int32_t order, uint8_t *d_inc, void *stream);

/* Algorithm 2 takes the intervals of x_1 as a list (Sec. 2.2); this is vx_csf_eval_level with
 * an explicit interval list per axis instead of the regular grid: a depth-j node labelled t
 * (j = 1..k) stands for [d_xlo[j-1][t], d_xhi[j-1][t]] (binary64, device, caller-owned,
 * nx[j-1] >= 2^level entries each, lo <= hi; the CSF's level only bounds its labels).  Test
 * hook for evaluations on point sets that are not grids: with X_j = {[1,1], [-1,-1]} a
 * multilinear polynomial gives the Walsh-Hadamard transform of its coefficients (the real
 * special case of the DFT identity of Sec. 3.1).  Outputs and modes as vx_csf_eval_level;
 * the binary32 modes take the interval ends rounded outward. */
int vx_csf_eval_grid(const vx_system *sys, const vx_csf *csf, const double *const *d_xlo,
                     const double *const *d_xhi, const int64_t *nx, int32_t mode, double *d_lo,
                     double *d_hi, uint8_t *d_keep, void *stream);

/* Level evaluation that allocates nothing, for callers that cannot allocate device memory
 * while they run: a host framework that owns the device's memory as a fixed budget (where an
 * allocation by a library would fail or upset its accounting), or a latency-bound loop that
 * must not risk the synchronisation or the out-of-memory failure an allocation can bring.
 * The paper has no counterpart; this is vx_csf_eval_level in VX_FP64 or VX_FP32_MIDRAD (the
 * same kernels, the same outputs, bit for bit) with its scratch, the partial-evaluation
 * blocks of depths 1..k-1, taken from one array of VX_STATIC_SCRATCH_BYTES bytes of device
 * memory that the library declares statically: every device that loads the library holds it
 * until the process exits.  The caller passes inputs and outputs as for vx_csf_eval_level.
 *   - VX_ECAPACITY (with the needed size in vx_last_error) when the blocks do not fit: at most
 *     sum over polynomials and depths d < k of N_d * M_d * (16 bytes for VX_FP64, 8 for
 *     VX_FP32_MIDRAD), each block rounded up to 256 bytes; VX_EINVAL for VX_FP32.
 *   - No cudaMalloc, cudaFree or allocating library routine is called.  The first call on a
 *     device looks up the array's device address (cudaGetSymbolAddress) with that device
 *     current and keeps it for the process (a lock guards concurrent first calls); make that
 *     first call before any stream capture.  The address belongs to the device's context:
 *     after a cudaDeviceReset of that device, do not call this entry point on it again.
 *   - Like vx_csf_eval_level, the first evaluation of each new level shape times the kernels'
 *     launch variants on `stream` (events and a stream synchronisation) unless the variant
 *     choice is fixed with vx_autotune (mode 0, a forced variant, or a tuner cache file that
 *     already holds the shape).
 *   - Every call shares the array and leaves its contents behind; each block read is written
 *     earlier in the same call, so nothing needs clearing, but calls that overlap on the GPU
 *     (other streams, other host threads) race on it and must be serialised by the caller.
 *   - Returns once the evaluation is complete (synchronises `stream`). */
#define VX_STATIC_SCRATCH_BYTES (64ull << 20)
int vx_csf_eval_level_static(const vx_system *sys, const vx_csf *csf, const double *h_domain,
                             int32_t mode, double *d_lo, double *d_hi, uint8_t *d_keep,
                             void *stream);

/* Algorithm 3, one step: drops the leaves with d_keep[i] == 0 (and the inner nodes left
 * without leaves), bisects every remaining box 2^k ways and returns the CSF of level+1 (its
 * leaves are the 2^k children of each kept box, lexicographically ordered).  No sort: each
 * new node's position follows from the kept tree's counts.  An empty keep set gives an
 * empty CSF. */
int vx_csf_subdivide(const vx_csf *in, const uint8_t *d_keep, void *stream, vx_csf **out);
/* The kept leaves of `in` as a CSF of the same level (stable: leaf order preserved).
 * d_index (nullable, [N_k(out)]) receives for each kept leaf its leaf index in `in`. */
int vx_csf_compact(const vx_csf *in, const uint8_t *d_keep, int32_t *d_index, void *stream,
                   vx_csf **out);

/* Algorithm 3 to `depth` on a device-resident system: tests levels 0..depth with C0 and
 * returns the survivors of level `depth` (a box of the finest grid is returned iff every
 * polynomial's interval value on it contains 0, in the arithmetic `opts` selects for that
 * level; with VX_FP64 throughout, or VX_FP32_MIDRAD with fp64_final, this is exactly the
 * VX_FP64 set).  opts may be NULL (VX_FP64).  Ordered on `stream`; returns once the
 * result is complete. */
int vx_enclose_system(const vx_system *sys, const double *h_domain, int32_t depth,
                      const vx_opts *opts, void *stream, vx_result **out);
/* Algorithm 3 with the set S initialised to the boxes of `start` (a CSF of level l0 <= depth,
 * borrowed): levels l0..depth are tested and the survivors of level `depth` returned.  The
 * survivors of the finest level do not depend on how coarser levels were pruned (interval
 * Horner with outward rounding is inclusion-isotone on an exact grid), so starting from a
 * subset of a level gives exactly the full run's survivors that descend from that subset:
 * independent x_1-slabs of one problem can run on different GPUs.  Statistics of levels below
 * l0 are zero. */
int vx_enclose_from(const vx_system *sys, const vx_csf *start, const double *h_domain,
                    int32_t depth, const vx_opts *opts, void *stream, vx_result **out);
/* The same from host polynomials: packs and uploads them and runs on a private stream; the
 * result's boxes reach the host through vx_result_boxes (tuples) or vx_result_box_codes
 * (grid indices), each copying on its first call. */
int vx_enclose(const vx_poly *F_list, int32_t npoly, const double *h_domain, int32_t depth,
               const vx_opts *opts, vx_result **out);

/* Algorithm 3 on nsys independent systems (each its own k, polynomials, domain and depth):
 * systems[i] points to npoly[i] polynomials, its domain is the next 2 k_i doubles of
 * `domains` (systems in order), depths[i] its depth; out[i] receives its result (its boxes
 * on the device as for vx_enclose_system; vx_result_boxes copies them).  The systems with the same k
 * run together as one forest of CSF trees per level: each depth of a level is one launch over
 * every tree's nodes (each with its own polynomials and grid), the binary64 re-evaluations of
 * VX_FP32 (error band) and VX_FP32_MIDRAD (tight boxes with fp64_recheck; a system's last
 * level with fp64_final) run as one forest too, and the prune and bisection are one scan over
 * the forest, so a level costs one host synchronisation per prune for all the systems.  Each
 * result is the one vx_enclose gives for that system alone; its elapsed time is its group's.
 * nworkers is not used.  On failure every out[i] is NULL. */
int vx_enclose_batch(const vx_poly *const *systems, const int32_t *npoly, const double *domains,
                     const int32_t *depths, int32_t nsys, const vx_opts *opts, int32_t nworkers,
                     vx_result **out);

/* Autotuner of the evaluation kernels (not in the paper).  Each stage and leaf launch has a
 * few variants with identical outputs (one or two boxes per thread, numbers of fibre groups,
 * CTA sizes, the parents' blocks staged in shared memory or not, the leaf pairs that the first
 * polynomial excludes skipped by the others); with mode 1 (the default) the first launch of a shape (arithmetic, depth, node
 * counts and fibre length, bucketed) times every variant on its real data and keeps the
 * fastest for the later ones (that first launch synchronises its stream); mode 0 uses the
 * built-in heuristics.  cache_path (nullable): a text file of tuned shapes, read by this call
 * and appended to as shapes are tuned.  Mode 2 + v runs variant v of every launch that has
 * one (else variant 0), without timing: a test hook that exercises each variant (every
 * variant gives the same outputs).  vx_autotune_entries: shapes tuned so far;
 * vx_autotune_clear forgets them. */
int vx_autotune(int32_t mode, const char *cache_path);
int vx_autotune_entries(void);
void vx_autotune_clear(void);

/* ---- Dense full-grid levels on the tensor cores (k = 3) ------------------------------------
 * Property 1 (Sec. 1) writes a polynomial on a tensor grid as one contraction of its
 * coefficient tensor per variable.  A plan evaluates every box of a level (2^level boxes per
 * axis over the domain) of a trivariate system that way: per polynomial, a midpoint-radius
 * enclosure mode by mode (the midpoints by TF32 tensor-core contractions with the grid's
 * Vandermonde matrices, the radii by contractions of |midpoint| and radius with
 * ((|c|+r)^a - |c|^a) and (|c|+r)^a, every rounding charged to the radius).  That enclosure
 * contains the nested interval Horner enclosure of Algorithm 1 on every box, so the boxes it
 * keeps under C0 (Sec. 3.2: 0 in every polynomial's enclosure) are a superset of the boxes the
 * interval-Horner level keeps.  The paper has no tensor-core path; this is the dense case of
 * Algorithm 2 (every node of every depth present) recast as GEMMs.
 *
 * vx_dense_plan_create: builds every operand (the coefficient tensor as TF32 panels, the grid's
 * factor matrices) and the intermediates for `sys` (k = 3, degree <= 255 in x_3) at `level`
 * (5..12) on h_domain (the exact grids vx_csf_eval_level accepts).  Device memory: about
 * 4 (2^level)^2 ((d1+1)(d3+1) + 3 (d3+1) 2^level) bytes per polynomial, reported by
 * vx_dense_plan_bytes.  The plan borrows `sys`, which must outlive it.  Ordered on `stream`;
 * returns once the plan is ready. */
typedef struct vx_dense_plan vx_dense_plan;
int vx_dense_plan_create(const vx_system *sys, int32_t level, const double *h_domain,
                         void *stream, vx_dense_plan **out);
int vx_dense_plan_bytes(const vx_dense_plan *plan, int64_t *bytes);
void vx_dense_plan_free(vx_dense_plan *plan);
/* The superset as a bit mask (device, caller-owned, 2^(3 level) / 32 words): bit b of word w
 * is box i = 32 w + b, i = (t1 2^level + t2) 2^level + t3, set iff the box is kept.  Launches
 * only (3 per polynomial, no allocation, no synchronisation): the first call for a mask
 * address captures them as a CUDA graph, later calls replay it.  A plan serves one host
 * thread at a time.  A tensor-core wait that gave up is reported by the next vx_dense_level
 * or vx_dense_check_status. */
int vx_dense_prefilter(const vx_dense_plan *plan, uint32_t *d_mask, void *stream);
/* VX_ETIMEOUT if a bounded wait inside a tensor-core kernel gave up since the last check
 * (the outputs of that launch are not valid); synchronises `stream`. */
int vx_dense_check_status(void *stream);
/* Test hook: polynomial `poly`'s final midpoint and radius on every box (device, caller-owned,
 * [2^(3 level)] binary32 each, box order as above).  Every value of the polynomial on box i
 * lies in [d_mid[i] - d_rad[i], d_mid[i] + d_rad[i]]. */
int vx_dense_values(const vx_dense_plan *plan, int32_t poly, float *d_mid, float *d_rad,
                    void *stream);
/* The level decided exactly: the prefilter, then the surviving boxes as a CSF evaluated by
 * vx_csf_eval_level's path in opts->mode (VX_FP64, or VX_FP32, which decides every box as
 * VX_FP64 does; VX_FP32_MIDRAD gives a superset).  d_keep (device, caller-owned,
 * [2^(3 level)] bytes, box order as above) equals vx_csf_eval_level's keep on the full grid
 * of the level in that mode; *n_survivors (nullable) receives the prefilter's count.
 * opts may be NULL (VX_FP32).  Returns once complete. */
int vx_dense_level(const vx_dense_plan *plan, const vx_opts *opts, uint8_t *d_keep,
                   int64_t *n_survivors, void *stream);

/* The surviving boxes: *n tuples of k int32 grid indices at level `depth`, lexicographic,
 * in host memory owned by the result (copied from the device on first call). */
int vx_result_boxes(vx_result *res, int64_t *n, const int32_t **h_tuples);
/* With opts.c1: the boxes C1 certified, *n of them, ordered by level, then lexicographic:
 * h_levels[i] the level of box i and h_tuples[i*k ..] its k grid indices at that level; host
 * memory owned by the result (copied from the device on first call). */
int vx_result_included(vx_result *res, int64_t *n, const int32_t **h_levels,
                       const int32_t **h_tuples);
/* The surviving boxes in compact form: *n codes, each a box's index in the full level-`depth`
 * grid with x_1 most significant (sum_i t_i 2^(depth (k-1-i))), ascending (the lexicographic
 * order of the tuples); *code_bytes = 4 when k * depth <= 32 (uint32 codes), else 8 (uint64).
 * Host memory owned by the result (copied from the device on first call): a third of the
 * tuples' bytes at k = 3, for callers that move results off the GPU in bulk. */
int vx_result_box_codes(vx_result *res, int64_t *n, int32_t *code_bytes, const void **h_codes);
/* The survivors as a device CSF owned by the result (valid until vx_result_free); for an
 * enclosure run in x_1 ranges (opts.max_level_boxes) the ranges' trees joined into one on the
 * first call, VX_EOVERFLOW if they hold more than 2^31 - 1 boxes. */
int vx_result_csf(const vx_result *res, const vx_csf **csf);
/* Per-level statistics, levels 0..depth: h_tested[l] = |S_l| boxes evaluated, h_kept[l]
 * survivors, h_nodes[l*k + j-1] = N_j(S_l), h_recheck[l] = boxes re-decided beyond the level's
 * first arithmetic (VX_FP32: the binary32 error band, decided by the float-pair tier and what
 * it leaves by VX_FP64; VX_FP32_MIDRAD with fp64_recheck: the tight boxes, in VX_FP64),
 * h_madds[l] = interval multiply-adds of the level (Theorem 1's count: sum over polynomials
 * and depths j of N_j (M_{j-1} - M_j)), plus those of the re-evaluations.
 * Any pointer may be NULL; *nlevels = depth + 1. */
int vx_result_stats(const vx_result *res, int32_t *nlevels, int64_t *h_tested, int64_t *h_kept,
                    int64_t *h_nodes, int64_t *h_recheck, int64_t *h_madds);
/* Of the boxes h_recheck counts, those decided in VX_FP64, per level 0..depth (VX_FP32: the
 * boxes the float-pair tier leaves undecided; otherwise all of them). */
int vx_result_recheck64(const vx_result *res, int64_t *h_per_level);
/* Kernel timing (opts.timing != 0): for kernel kind i < *nkinds: h_ms[i] summed CUDA-event
 * time, h_launches[i] launches, h_work[i] algorithmic work (interval multiply-adds for the
 * evaluation kernels, bytes for the integer kernels).  vx_kernel_kind_name(i) names kind i. */
int vx_result_timing(const vx_result *res, int32_t *nkinds, double *h_ms, int64_t *h_launches,
                     int64_t *h_work);
const char *vx_kernel_kind_name(int32_t kind);
/* Wall time of the level loop on the stream (CUDA events), in milliseconds. */
int vx_result_elapsed_ms(const vx_result *res, double *ms);
void vx_result_free(vx_result *res);

#ifdef __cplusplus
}
#endif

#endif /* VX_H */
