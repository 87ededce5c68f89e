// vx_eval.cu -- level evaluation: Algorithm 2 (EvaluationCSF) run level-synchronously.
//
// Algorithm 2 recurses node by node; here each CSF depth d is one launch over all depth-d
// nodes at once.  A depth-d node runs stage d of the packed polynomial: Algorithm 1 (Horner)
// in x_{d+1} on its own interval, once per fibre, on the input block its parent produced
// (the coefficient tensor itself at depth 0), and writes its own block for its children.
// The leaves (depth k-1) run the last stage, a single fibre, and apply criterion C0 of
// Sec. 3.2 (drop the box iff 0 is outside the value of some polynomial).  Per box this is
// exactly nested Horner: the same operations in the same order, so a depth-d block depends
// only on the intervals along the path and not on which other boxes share the tree.
//
// Two arithmetics share the kernels through a policy class:
//   A64: binary64 intervals [lo, hi] with __dmul_rd/__dmul_ru/__dadd_rd/__dadd_ru.  The
//        product J*X uses the sign of X (fixed per node) and of J's endpoints to pick the one
//        endpoint product that is the min (max); RD/RU are monotone, so this is the same
//        double as the min (max) of the four directed products.  Signs are read from the
//        high word (integer ops), keeping the scarce FP64 pipe for the 4 arithmetic ops.
//   A32: binary32 midpoint-radius <m, r>.  One Horner step J*X + A gives
//          m = RN(Jm*Xm + Am)
//          r = RU(Jr*RU(|Xm|+Xr) + Ar) then RU(|Jm|*Xr + r) then RU(2^-24*|m| + r)
//        which bounds |j*x + a - m| for all j in J, x in X, a in A: the exact distance is at
//        most Jr(|Xm|+Xr) + |Jm|Xr + Ar, and rounding m to nearest adds at most 2^-24|m| plus
//        2^-149 below the normal range, which every coefficient radius already carries
//        (it is added when a block is stored).  Inf or NaN never excludes a box.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include "vx_internal.cuh"

namespace vx {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double sel_min(double a, double b) { return (b < a) ? b : a; }
__device__ __forceinline__ double sel_max(double a, double b) { return (b > a) ? b : a; }
__device__ __forceinline__ bool sign_clear(double v) { return __double2hiint(v) >= 0; }

struct A64 {
  using V = double2;  // .x = lo, .y = hi
  struct X {
    double l, h;
    int cls;  // 1: X >= 0, -1: X <= 0, 0: X straddles 0
  };
  static __device__ __forceinline__ X box(const AxisGrid &g, int32_t t) {
    X x;
    x.l = __dadd_rn(g.lo, __dmul_rn((double)t, g.w));  // exact on accepted domains
    x.h = __dadd_rn(g.lo, __dmul_rn((double)t + 1.0, g.w));
    x.cls = (x.l >= 0.0) ? 1 : ((x.h <= 0.0) ? -1 : 0);
    return x;
  }
  static __device__ __forceinline__ V muladd(V J, const X &x, V A) {
    double lo, hi;
    if (x.cls > 0) {
      lo = __dmul_rd(J.x, sign_clear(J.x) ? x.l : x.h);
      hi = __dmul_ru(J.y, sign_clear(J.y) ? x.h : x.l);
    } else if (x.cls < 0) {
      lo = __dmul_rd(J.y, sign_clear(J.y) ? x.l : x.h);
      hi = __dmul_ru(J.x, sign_clear(J.x) ? x.h : x.l);
    } else {
      lo = sel_min(sel_min(__dmul_rd(J.x, x.l), __dmul_rd(J.x, x.h)),
                   sel_min(__dmul_rd(J.y, x.l), __dmul_rd(J.y, x.h)));
      hi = sel_max(sel_max(__dmul_ru(J.x, x.l), __dmul_ru(J.x, x.h)),
                   sel_max(__dmul_ru(J.y, x.l), __dmul_ru(J.y, x.h)));
    }
    return make_double2(__dadd_rd(lo, A.x), __dadd_ru(hi, A.y));
  }
  static __device__ __forceinline__ V store(V J) { return J; }
  static __device__ __forceinline__ bool contains0(V J) { return !(J.x > 0.0 || J.y < 0.0); }
  static __device__ __forceinline__ double lo(V J) { return J.x; }
  static __device__ __forceinline__ double hi(V J) { return J.y; }
  static __device__ __forceinline__ bool tight(V, float) { return false; }
  static __host__ __device__ __forceinline__ const V *coef(const PolyDev &p) { return p.c64; }
};

constexpr float kU32 = 5.9604644775390625e-08f;  // 2^-24, unit roundoff of binary32
constexpr float kEta32 = 1.40129846e-45f;        // 2^-149, smallest positive binary32

struct A32 {
  using V = float2;  // .x = m, .y = r
  struct X {
    float m, r, a;  // a >= |m| + r
  };
  static __device__ __forceinline__ X box(const AxisGrid &g, int32_t t) {
    X x;
    if (g.fexact) {
      // every half-grid point is a binary32: centre and half-width are exact
      x.m = __fmaf_rn((float)t + 0.5f, g.fw, g.flo);
      x.r = 0.5f * g.fw;
    } else {
      double l = __dadd_rn(g.lo, __dmul_rn((double)t, g.w));
      double h = __dadd_rn(g.lo, __dmul_rn((double)t + 1.0, g.w));
      x.m = __double2float_rn(0.5 * l + 0.5 * h);
      double dm = (double)x.m;
      x.r = __double2float_ru(fmax(__dadd_ru(h, -dm), __dadd_ru(dm, -l)));
    }
    x.a = __fadd_ru(fabsf(x.m), x.r);
    return x;
  }
  static __device__ __forceinline__ V muladd(V J, const X &x, V A) {
    float m = __fmaf_rn(J.x, x.m, A.x);
    float r = __fmaf_ru(J.y, x.a, A.y);
    r = __fmaf_ru(fabsf(J.x), x.r, r);
    r = __fmaf_ru(kU32, fabsf(m), r);
    return make_float2(m, r);
  }
  static __device__ __forceinline__ V store(V J) { return make_float2(J.x, __fadd_ru(J.y, kEta32)); }
  static __device__ __forceinline__ bool contains0(V J) { return !(fabsf(J.x) > J.y); }
  static __device__ __forceinline__ double lo(V J) { return __dadd_rd((double)J.x, -(double)J.y); }
  static __device__ __forceinline__ double hi(V J) { return __dadd_ru((double)J.x, (double)J.y); }
  static __device__ __forceinline__ bool tight(V J, float theta) {
    return fabsf(J.x) >= theta * J.y;
  }
  static __host__ __device__ __forceinline__ const V *coef(const PolyDev &p) { return p.c32; }
};

// Stage d < k-1 on every depth-d node: item = (node, fibre), fibres fastest so that a warp
// reads consecutive entries of one row of the parent's block at each Horner step.
template <class AR>
__global__ void __launch_bounds__(kThreads)
    k_stage(const StageDev st, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
            const typename AR::V *__restrict__ in, typename AR::V *__restrict__ out,
            int64_t nnodes, AxisGrid g) {
  using V = typename AR::V;
  extern __shared__ int32_t s_rowoff[];
  for (int i = threadIdx.x; i <= st.maxlen; i += blockDim.x) s_rowoff[i] = st.rowoff[i];
  __syncthreads();
  const int64_t nitems = nnodes * st.nfib;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems; i += stride) {
    const int64_t node = i / st.nfib;
    const int fib = (int)(i - node * st.nfib);
    const V *base = par ? in + (int64_t)__ldg(par + node) * st.blk_in : in;
    const typename AR::X x = AR::box(g, __ldg(lab + node));
    const int L = __ldg(st.fiblen + fib);
    V J = base[s_rowoff[L - 1] + fib];
    for (int a = L - 2; a >= 0; --a) J = AR::muladd(J, x, base[s_rowoff[a] + fib]);
    out[node * st.blk_out + __ldg(st.outpos + fib)] = AR::store(J);
  }
}

struct LeafArgs {
  const void *in[VX_MAXPOLY];  // parent blocks per polynomial (the coefficients when k == 1)
  int64_t blk[VX_MAXPOLY];
  int32_t len[VX_MAXPOLY];
};

// Last stage on every leaf: one Horner per polynomial, then C0.
template <class AR>
__global__ void __launch_bounds__(kThreads)
    k_leaf(LeafArgs A, int npoly, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
           int64_t nleaves, AxisGrid g, uint8_t *__restrict__ keep, double *__restrict__ lo,
           double *__restrict__ hi, uint8_t *__restrict__ tight, float theta) {
  using V = typename AR::V;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += stride) {
    const typename AR::X x = AR::box(g, __ldg(lab + i));
    const int64_t p = par ? (int64_t)__ldg(par + i) : 0;
    bool kp = true, tg = false;
    for (int f = 0; f < npoly; ++f) {
      const V *base = (const V *)A.in[f] + p * A.blk[f];
      const int L = A.len[f];
      V J = base[L - 1];
      for (int a = L - 2; a >= 0; --a) J = AR::muladd(J, x, base[a]);
      if (lo) {
        lo[(int64_t)f * nleaves + i] = AR::lo(J);
        hi[(int64_t)f * nleaves + i] = AR::hi(J);
      }
      kp = kp && AR::contains0(J);
      tg = tg || AR::tight(J, theta);
    }
    keep[i] = kp ? 1 : 0;
    if (tight) tight[i] = (kp && tg) ? 1 : 0;
  }
}

bool tracing() {
  static int on = -1;
  if (on < 0) on = std::getenv("VX_TRACE") ? 1 : 0;
  return on == 1;
}

int grid_for(int64_t items) {
  int64_t b = (items + kThreads - 1) / kThreads;
  const int64_t cap = 152 * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

template <class AR>
int eval_level_t(const SysDev &sys, const CsfView &c, const LevelGrid &grid, double *d_lo,
                 double *d_hi, uint8_t *d_keep, uint8_t *d_tight, float theta, cudaStream_t s,
                 Timer *tm, int64_t *madds_out, int kind0) {
  using V = typename AR::V;
  const int k = sys.k;
  const int64_t nleaves = c.N[k - 1];
  int64_t madds = 0;
  if (nleaves == 0) {
    if (madds_out) *madds_out = 0;
    return VX_OK;
  }
  // partial-polynomial blocks of depths 0..k-2, one allocation per polynomial
  void *mem[VX_MAXPOLY] = {nullptr};
  V *buf[VX_MAXPOLY][VX_KMAX] = {{nullptr}};
  int rc = VX_OK;
  for (int f = 0; f < sys.npoly && rc == VX_OK; ++f) {
    size_t total = 0;
    for (int d = 0; d + 1 < k; ++d) total += (size_t)c.N[d] * sys.p[f].st[d].blk_out;
    if (total == 0) continue;
    rc = dmalloc(&mem[f], total * sizeof(V), s);
    size_t off = 0;
    for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
      buf[f][d] = (V *)mem[f] + off;
      off += (size_t)c.N[d] * sys.p[f].st[d].blk_out;
    }
  }
  for (int f = 0; f < sys.npoly && rc == VX_OK; ++f) {
    for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
      const StageDev &st = sys.p[f].st[d];
      const int64_t items = c.N[d] * st.nfib;
      const int64_t w = c.N[d] * (st.blk_in - st.nfib);
      madds += w;
      if (tm && tm->on) rc = tm->begin(d == 0 ? kind0 : kind0 + 1, w);
      if (rc != VX_OK) break;
      if (tracing())
        std::fprintf(stderr, "[vx] stage %d launch poly %d items=%lld smem=%d\n", d, f,
                     (long long)items, (int)((st.maxlen + 1) * sizeof(int32_t)));
      const V *in = d == 0 ? AR::coef(sys.p[f]) : buf[f][d - 1];
      k_stage<AR><<<grid_for(items), kThreads, (st.maxlen + 1) * sizeof(int32_t), s>>>(
          st, c.lab[d], d == 0 ? nullptr : c.par[d], in, buf[f][d], c.N[d], grid.ax[d]);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        set_error("stage kernel launch failed: %s", cudaGetErrorString(e));
        rc = VX_ECUDA;
        break;
      }
      if (tm && tm->on) rc = tm->end();
    }
  }
  if (rc == VX_OK) {
    LeafArgs A;
    int64_t wl = 0;
    for (int f = 0; f < sys.npoly; ++f) {
      const StageDev &st = sys.p[f].st[k - 1];
      A.in[f] = k == 1 ? (const void *)AR::coef(sys.p[f]) : (const void *)buf[f][k - 2];
      A.blk[f] = k == 1 ? 0 : st.blk_in;
      A.len[f] = st.maxlen;
      wl += nleaves * (st.blk_in - 1);
    }
    madds += wl;
    if (tm && tm->on) rc = tm->begin(kind0 + 2, wl);
    if (tracing())
      std::fprintf(stderr, "[vx] leaf launch k=%d npoly=%d n=%lld grid=%d len0=%d\n", k,
                   sys.npoly, (long long)nleaves, grid_for(nleaves), A.len[0]);
    if (rc == VX_OK) {
      k_leaf<AR><<<grid_for(nleaves), kThreads, 0, s>>>(A, sys.npoly, c.lab[k - 1],
                                                        k == 1 ? nullptr : c.par[k - 1], nleaves,
                                                        grid.ax[k - 1], d_keep, d_lo, d_hi,
                                                        d_tight, theta);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        set_error("leaf kernel launch failed: %s", cudaGetErrorString(e));
        rc = VX_ECUDA;
      }
      if (rc == VX_OK && tm && tm->on) rc = tm->end();
    }
  }
  for (int f = 0; f < sys.npoly; ++f) dfree(mem[f], s);
  if (madds_out) *madds_out = madds;
  return rc;
}

}  // namespace

int eval_level(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, int mode,
               double *d_lo, double *d_hi, uint8_t *d_keep, cudaStream_t s, Timer *tm,
               int64_t *madds_out) {
  if (mode == VX_FP64)
    return eval_level_t<A64>(sys, csf, grid, d_lo, d_hi, d_keep, nullptr, 0.f, s, tm, madds_out,
                             KK_STAGE0);
  return eval_level_t<A32>(sys, csf, grid, d_lo, d_hi, d_keep, nullptr, 0.f, s, tm, madds_out,
                           KK_STAGE0_F32);
}

int eval_level_tight(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, float theta,
                     uint8_t *d_keep, uint8_t *d_tight, cudaStream_t s, Timer *tm,
                     int64_t *madds_out) {
  return eval_level_t<A32>(sys, csf, grid, nullptr, nullptr, d_keep, d_tight, theta, s, tm,
                           madds_out, KK_STAGE0_F32);
}

}  // namespace vx
