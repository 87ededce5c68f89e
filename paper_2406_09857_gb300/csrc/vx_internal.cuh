// vx_internal.cuh -- shared declarations of libvx (device structs, interval arithmetic,
// error handling).  Not part of the public ABI (that is include/vx.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "vx.h"

namespace vx {

// ---------------------------------------------------------------------------------------
// Errors: every entry point returns a VX_* code; the message goes to a thread-local buffer.
// ---------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

#define VX_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::vx::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                      __LINE__);                                                          \
      return VX_ECUDA;                                                                    \
    }                                                                                     \
  } while (0)

#define VX_CHECK(x)                  \
  do {                               \
    int rc_ = (x);                   \
    if (rc_ != VX_OK) return rc_;    \
  } while (0)

#define VX_LAUNCH_CHECK() VX_CUDA(cudaGetLastError())

// Counts the kernels this library launches (process-wide, all threads).
void note_launch(int n = 1);

// Streaming multiprocessors of the current device (cudaDevAttrMultiProcessorCount, read once
// per device); grid sizes are multiples of it.
int sm_count();

// Stream-ordered device memory (the device's default memory pool, kept cached).
int dmalloc(void **p, size_t bytes, cudaStream_t s);
void dfree(void *p, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// Packed polynomial (Sec. 2.1, "Representing a Multivariate Polynomial", re-laid out for the
// device).  Stage s (0-based) evaluates x_{s+1}: it runs Algorithm 1 once per fibre, a fibre
// being one monomial m in x_{s+2}..x_k with coefficients indexed by the exponent a of
// x_{s+1}, a = 0..len(m)-1 (missing exponents below the highest are zero coefficients).
// Fibres are sorted by decreasing length, so row a of the stage input holds the fibres with
// len > a, i.e. fibres 0..rowcount(a)-1, at rowoff[a] .. rowoff[a+1]-1: consecutive threads
// on consecutive fibres read consecutive addresses at every Horner step.  The value of fibre
// f is written at outpos[f] of the next stage's input block.
// ---------------------------------------------------------------------------------------
// A stage whose parent blocks are staged in shared memory (k_stage_tma*) reads its input
// fibre-major instead: fibre f's entries a = 0..len-1 at fiboff[f] + a, so that a Horner walks
// consecutive entries and a group of consecutive fibres is one contiguous range; its producer
// then writes fibre f's value at outpos_fm[f] instead of outpos[f].
struct StageDev {
  int32_t nfib, maxlen;
  int64_t blk_in;   // entries of one input block of this stage
  int64_t blk_out;  // entries of one output block (= next stage's blk_in; 1 at the last stage)
  const int32_t *rowoff;     // [maxlen + 1]
  const int32_t *fiblen;     // [nfib]
  const int32_t *outpos;     // [nfib] (unused at the last stage)
  const int32_t *fiboff;     // [nfib + 1] fibre-major offsets of this stage's input
  const int32_t *outpos_fm;  // [nfib] position in the next stage's fibre-major input
};

struct PolyDev {
  StageDev st[VX_KMAX];
  const double2 *c64;  // stage-0 input block as degenerate intervals (lo = hi = coefficient)
  const float2 *c32;   // stage-0 input block as <m, r> binary32 midpoint-radius pairs
  const float4 *c32c;  // stage-0 input block as binary32 [RD(c), RU(c)] with error bound
  // the three blocks above fibre-major (st[0].fiboff): a stage-0 Horner walks consecutive
  // entries instead of one row (a cache line) per step
  const double2 *c64_fm;
  const float2 *c32_fm;
  const float4 *c32c_fm;
  const float4 *cp;    // stage-0 input block as float pairs (lo_h, lo_l, -hi_h, -hi_l) ...
  const float *ep;     // ... and their error bounds (eval_level_pair)
  const float4 *cp_fm;  // the same two fibre-major (st[0].fiboff)
  const float *ep_fm;
};

struct SysDev {
  int32_t k, npoly;
  PolyDev p[VX_MAXPOLY];
  int8_t rel[VX_MAXPOLY];  // relation of each polynomial: VX_EQ, VX_LE, VX_GE, VX_LT, VX_GT
};

// One axis of one grid level: box t is [lo + t*w, lo + (t+1)*w] (exact on accepted domains).
struct AxisGrid {
  double lo, w;
  float flo, fw;    // the same in binary32 when every half-grid point is a binary32
  int32_t fexact;   // 1 if flo/fw describe the grid exactly
  // explicit intervals (device arrays, label t -> [xlo[t], xhi[t]]) instead of the regular
  // grid when non-null; fexact is 0 then
  const double *xlo, *xhi;
  // nonzero: box t stands for a point of it, as the point interval [x, x]: 1 its centre
  // x = lo + (t + 1/2) w, 2 its lower end lo + t w, 3 its upper end lo + (t + 1) w
  int32_t point;
};

struct LevelGrid {
  AxisGrid ax[VX_KMAX];
};

// ---------------------------------------------------------------------------------------
// Device CSF of box indices (Sec. 2.1, "Representing a Set of Boxes").  Depth d (0-based)
// holds N[d] nodes: label lab[d][i] (grid index along x_{d+1}), parent par[d][i] (d >= 1,
// node index at depth d-1) and, for d < k-1, child range ptr[d][i] .. ptr[d][i+1]-1.
// ---------------------------------------------------------------------------------------
struct CsfView {
  int32_t k, level;
  int64_t N[VX_KMAX];
  int32_t *lab[VX_KMAX];
  int32_t *par[VX_KMAX];
  int32_t *ptr[VX_KMAX];
};

// ---------------------------------------------------------------------------------------
// Kernel timing (CUDA events around launches when enabled).
// ---------------------------------------------------------------------------------------
enum KernelKind {
  KK_STAGE0 = 0,   // depth-1 partial evaluation (reads the coefficient tensor)
  KK_STAGEJ,       // depth-j partial evaluation, 1 < j < k
  KK_LEAF,         // leaf Horner + C0 test
  KK_STAGE0_F32,
  KK_STAGEJ_F32,
  KK_LEAF_F32,
  KK_STAGE0_F32C,
  KK_STAGEJ_F32C,
  KK_LEAF_F32C,
  // The integer phases' work is their algorithmic bytes: each input array read once and each
  // output array written once (node counts N_d, total = sum N_d, kept nk_d, new newN_d).
  KK_CSF_BUILD,    // scans of csf_build: the tuples read, the tree's arrays written
  KK_PRUNE,        // keep propagation and rank scan: keep + ptr read, flags + ranks written
  KK_SPLIT,        // 2^k split and rebuild: flags + ranks read, kept nodes' arrays read, new
                   // nodes' arrays written
  KK_COMPACT,      // stable compaction: flags + ranks read, kept nodes' arrays read and written
  KK_RECHECK,      // selection of the boxes to re-evaluate: flags read, their indices written
  KK_STAGE0_PAIR,  // the float-pair tier (eval_level_pair) on the binary32 path's error band
  KK_STAGEJ_PAIR,
  KK_LEAF_PAIR,
  KK_COUNT
};

struct Timer {
  bool on = false;
  cudaStream_t stream = nullptr;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
    int64_t work;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double ms[KK_COUNT] = {0};
  int64_t launches[KK_COUNT] = {0};
  int64_t work[KK_COUNT] = {0};
  int begin(int kind, int64_t work);  // records the start event on `stream`
  int end();                          // records the stop event of the last begin()
  // adds to the work of the last begin() (for counts known only once its kernels ran)
  void add_work(int64_t w) {
    if (!pending.empty()) pending.back().work += w;
  }
  int collect();                      // synchronises and folds pending pairs into the sums
  void release();
};

// Launcher (vx_eval.cu): one level in one arithmetic.  d_keep[i] = 0 iff the box is
// excluded; d_flag (nullable) marks the kept boxes to re-evaluate in binary64: for
// ARITH_F32_MIDRAD those with |m| >= theta r for some polynomial, for ARITH_F32_CERT those
// inside the error band of some polynomial.
enum Arith { ARITH_F64 = 0, ARITH_F32_MIDRAD = 1, ARITH_F32_CERT = 2 };
// The float-pair tier: every interval end as an unevaluated sum of two binary32 numbers (about
// 48 bits) with a bound on its distance to the binary64 path's end, on grids whose box ends are
// binary32 numbers.  keep[i] = 0 / 1 where the binary64 path surely excludes / keeps leaf i;
// flag[i] = 1 where the tier cannot tell (keep[i] is then 1), to be decided in binary64.
int eval_level_pair(const SysDev &sys, const CsfView &csf, const LevelGrid &grid,
                    uint8_t *d_keep, uint8_t *d_flag, cudaStream_t s, Timer *tm,
                    int64_t *madds_out);
int eval_level_raw(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, int arith,
                   double *d_lo, double *d_hi, uint8_t *d_keep, uint8_t *d_flag, float theta,
                   cudaStream_t s, Timer *tm, int64_t *madds_out);
// The same without allocating (ARITH_F64 or ARITH_F32_MIDRAD): the blocks are carved from the
// library's fixed device array; VX_ECAPACITY if they do not fit in VX_STATIC_SCRATCH_BYTES.
int eval_level_static(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, int arith,
                      double *d_lo, double *d_hi, uint8_t *d_keep, cudaStream_t s);
// One level of a forest (the trees of many systems with the same k, one after another at
// every depth; tree s owns depth-d nodes off[d*(S+1)+s] .. off[d*(S+1)+s+1]-1).  d_trees and
// h_trees: the same table on the device and the host; h_off the host copy of d_off.
struct ForestTree {
  SysDev dev;
  AxisGrid ax[VX_KMAX];  // the level's grid of this tree's system
};
int eval_forest(int arith, const ForestTree *d_trees, const ForestTree *h_trees,
                const int64_t *d_off, const int64_t *h_off, int S, const CsfView &c,
                uint8_t *keep, uint8_t *flag, float theta, cudaStream_t s, int64_t *madds);
// The Taylor form of order m (Def. 3) of one polynomial F on every leaf, in binary64: tsys
// holds G_a = d^a F / a! for the multi-indices alpha[0..npoly-1] (|a| <= m, lexicographic);
// keep = C0 on T for the relation rel (first = 1) or keep &= that (first = 0); d_lo/d_hi
// (nullable) receive T;
// d_inc (nullable, m >= 2) receives the inclusion criterion C1 on the Taylor form.  d_flag
// non-null: the certified binary32 arithmetic (decisions as binary64 takes them, except on the
// boxes flagged there (flag |= unsure), which the caller re-decides in binary64; d_lo/d_hi
// must then be null).
int eval_level_taylor(const SysDev &tsys, const int8_t (*alpha)[VX_KMAX], int m,
                      const CsfView &c, const LevelGrid &grid, uint8_t *d_keep, int first, int rel,
                      double *d_lo, double *d_hi, uint8_t *d_inc, uint8_t *d_flag, cudaStream_t s,
                      Timer *tm, int64_t *madds);
// The inclusion criterion C1 by vertex signs (Sec. 3.2) of the system's one polynomial on
// every leaf: each of the 2^k corners of the boxes is evaluated through the CSF in binary64
// (point intervals); d_inc[i] = 1 iff one corner is certified > 0 and another < 0.
int eval_c1_vertex(const SysDev &sys, const CsfView &c, const LevelGrid &grid, uint8_t *d_inc,
                   cudaStream_t s, Timer *tm, int64_t *madds);
// Reads (synchronising `s`) and clears the device status word that a kernel sets when a
// bounded wait gives up; *status != 0 means the last evaluations are not to be trusted.
int take_device_status(cudaStream_t s, int *status);
// Polls of a kernel's first bounded wait on the current device (< 0: the default).
int set_wait_polls(int64_t polls);
// Autotuner of the stage and leaf launch variants (vx_eval.cu): mode 0 = heuristic variants
// only, 1 = time the variants of each new shape and keep the fastest; path (nullable) = a text
// cache read now and appended to.
int set_autotune(int mode, const char *path);
int autotune_entries();
void autotune_clear();

// Integer kernels (vx_csf.cu).  Objects own one device allocation each.
struct CsfObj {
  CsfView v;
  void *mem = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
};
int csf_alloc(CsfObj *o, int k, int level, const int64_t *N, cudaStream_t s);
void csf_release(CsfObj *o);
int csf_build_dev(int k, int level, const int32_t *d_tuples, int64_t n, cudaStream_t s,
                  CsfObj *out, Timer *tm);
// split = 1: Algorithm 3's bisection (level + 1); split = 0: stable compaction (same level),
// writing the kept leaves' old indices to d_index when non-null.
// cap: the most nodes the output may have at any depth (VX_EOVERFLOW beyond it; at most
// INT32_MAX, the tree's index range).
// Where a compaction writes its kept leaves' grid-index codes (k_box_codes' codes, 4 bytes
// when k * level <= 32, else 8) as it places them: get(ctx, n, code_bytes, &p) is called once
// the kept count n is known and returns in p a device-addressable array of n codes (nullptr:
// none are written) or an error.
struct CodesSink {
  int (*get)(void *ctx, int64_t n, int code_bytes, void **d_codes);
  void *ctx;
};
int csf_prune(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
              cudaStream_t s, CsfObj *out, Timer *tm, int64_t cap = INT32_MAX,
              const CodesSink *sink = nullptr);
// Per depth-0 node (an x_1 slab) r, d_cnt[r] = the leaves under it with d_keep set.
int csf_root_counts(const CsfView &c, const uint8_t *d_keep, int64_t *d_cnt, cudaStream_t s);
// d_out[i] = d_keep[i] for the leaves under depth-0 nodes a .. b-1, 0 elsewhere.
int csf_keep_in_roots(const CsfView &c, const uint8_t *d_keep, int64_t a, int64_t b,
                      uint8_t *d_out, cudaStream_t s);
// The same on a forest of nseg trees stored one after another at every depth (tree s owns
// depth-d nodes d_seg_off[d*(nseg+1) + s] .. [.. + s + 1] - 1): d_seg_kept[d*(nseg+1) + s]
// receives the kept depth-d nodes of trees before s (s = nseg: all of them), and h_seg_kept
// (nullable, host) a copy of it, read with the kept totals in the one wait of the call.
int csf_prune_forest(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
                     const int64_t *d_seg_off, int nseg, int64_t *d_seg_kept, cudaStream_t s,
                     CsfObj *out, Timer *tm, int64_t *h_seg_kept = nullptr);
// Queues a copy of the device status word (bounded waits that gave up) into pinned host memory
// (read it after the stream's next synchronisation).
int queue_device_status(cudaStream_t s, int *h_pinned);
// A pinned status word of the calling host thread (null if it cannot be allocated).
int *status_word();
// The complete tree of grid level `level` (every box), filled directly.
int csf_full_grid_dev(int k, int level, cudaStream_t s, CsfObj *out);
// ptr[d][N[d]] = N[d+1] for every depth d < k-1.
int set_ptr_sentinels(const CsfView &v, cudaStream_t s);
int csf_tuples_dev(const CsfView &c, int32_t *d_tuples, cudaStream_t s);
// Each leaf's box as its index in the level's full grid (x_1 most significant), uint32 when
// k * level <= 32, else uint64.
int csf_box_codes_dev(const CsfView &c, void *d_codes, cudaStream_t s);
// Increasing indices i with d_flags[i] != 0 (device array owned by the caller, freed with
// dfree; synchronises `s` to learn the count).
int flag_indices(const uint8_t *d_flags, int64_t n, cudaStream_t s, int32_t **d_idx,
                 int64_t *count);
// Index tuples of the listed leaves, d_tuples[n][k].
int csf_tuples_of(const CsfView &c, const int32_t *d_idx, int64_t n, int32_t *d_tuples,
                  cudaStream_t s);
int scatter_keep(const int32_t *d_index, const uint8_t *d_sub_keep, int64_t n, uint8_t *d_keep,
                 cudaStream_t s);


// ---- dense full-grid levels on the tensor cores (vx_dense.cu), k = 3 ----------------------
struct DenseHostPoly {
  const int32_t *exps;  // [nterms][3]
  const double *coefs;
  int64_t nterms;
};
struct DensePlan;
int dense_plan_create(int npoly, const DenseHostPoly *polys, int level, const double *domain,
                      cudaStream_t s, DensePlan **out);
void dense_plan_free(DensePlan *p);
int64_t dense_plan_bytes(const DensePlan *p);
int dense_plan_level(const DensePlan *p);
int dense_prefilter(DensePlan *p, uint32_t *d_mask, cudaStream_t s);
int dense_values(const DensePlan *p, int f, float *d_mid, float *d_rad, cudaStream_t s);
int set_dense_wait_polls(int64_t polls);
int take_dense_status(cudaStream_t s, int *status);
int mask_tuples(const uint32_t *d_mask, int level, cudaStream_t s, int32_t **d_tuples,
                int64_t *n);
int scatter_keep_grid(const int32_t *d_tuples, int64_t n, int level, const uint8_t *d_keep,
                      uint8_t *d_out, cudaStream_t s);

}  // namespace vx
