// vx_eval.cu -- level evaluation: Algorithm 2 (EvaluationCSF) run level-synchronously.
//
// Algorithm 2 recurses node by node; here each CSF depth d is one launch over all depth-d
// nodes at once.  A depth-d node runs stage d of the packed polynomial: Algorithm 1 (Horner)
// in x_{d+1} on its own interval, once per fibre, on the block its parent produced (the
// coefficient tensor itself at depth 0), and writes its own block for its children.  The
// leaves (depth k-1) run the last stage, a single fibre, and apply criterion C0 of Sec. 3.2
// (drop the box iff 0 is outside the value of some polynomial).  Per box this is exactly
// nested Horner: the same operations in the same order, so a block depends only on the
// intervals along its path, not on which other boxes share the tree.
//
// Layout and mapping.  The blocks of depth d are stored entry-major, P_d[e][node], and a warp
// takes 32 consecutive nodes (one lane each) through the same fibres in lock-step: at every
// Horner step its lanes read entry e of their parents' blocks, which is one address when the
// lanes are siblings (a broadcast) and consecutive addresses otherwise, and they store
// consecutive addresses.  The fibres of a stage are dealt round-robin to G warps per node
// chunk (fibres are sorted by length, so the groups carry nearly equal work), G chosen so the
// launch fills the GPU even when a depth has few nodes.
//
// Three arithmetics share the kernels through a policy class:
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
//   A32C: binary32 approximations of the interval ends stored as (lo, -hi), so that both ends
//        of J*X + A come from one paired FMA rounded to nearest (lo' = min over the endpoint
//        pairs of RN(J_e*X_e + A.lo), the same for -hi'), plus an error bound E carried with
//        every pair.  The pair is not an enclosure by itself: E bounds |lo32 - lo*| +
//        |lo64 - lo*| (and the same for hi), where lo* is the exact (unrounded) interval Horner
//        value with the binary64 coefficients and lo64 what A64 computes.  One step gives
//          E' = RU(E_J * xmax(1+2^-27) + RU((2^-24+2^-46)*m' + E_A)),  m' = max(|lo'|,|hi'|):
//        the min over endpoint products is xmax-Lipschitz in J and 1-Lipschitz in A; the FMA
//        rounds once to nearest (< 2^-24 of its result); the binary64 path rounds the product
//        (< 2^-52 |J| xmax, which is below 2^-28 E_J xmax because every bound satisfies
//        E >= 2^-24 max(|lo|,|hi|)) and the sum (< 2^-52 of it); every stored E carries a
//        relative margin of 2^-40 and an absolute 2^-148 (results below the normal range, whose
//        rounding is absolute), which exceed the binary64 rounding of a term in terms of the
//        bound itself, so the induction closes.  Hence lo32 > E means
//        A64's lower end is > 0 (A64 excludes the box) and lo32 <= -E with hi32 >= E means
//        A64 keeps it: a box is decided exactly as A64 decides it, except inside the band of
//        width E, where A64 is run on it.  Boxes whose grid points are not binary32 (domains
//        that are not exact at binary32 precision) add the term 2^-23 m_J xmax explicitly.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>

#include "vx_internal.cuh"
#include "vx_ptx.cuh"

namespace vx {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;

// The binary64 endpoints of box t on an axis: the regular grid (exact on accepted domains) or
// the axis' explicit interval list.
__device__ __forceinline__ void endpoints(const AxisGrid &g, int32_t t, double &l, double &h) {
  if (g.point == 1) {
    l = h = __dadd_rn(g.lo, __dmul_rn((double)t + 0.5, g.w));  // exact on accepted grids
  } else if (g.point) {  // 2: the lower end, 3: the upper end, as a point interval
    l = h = __dadd_rn(g.lo, __dmul_rn((double)t + (g.point == 3 ? 1.0 : 0.0), g.w));
  } else if (g.xlo) {
    l = g.xlo[t];
    h = g.xhi[t];
  } else {
    l = __dadd_rn(g.lo, __dmul_rn((double)t, g.w));
    h = __dadd_rn(g.lo, __dmul_rn((double)t + 1.0, g.w));
  }
}

__device__ __forceinline__ double sel_min(double a, double b) { return (b < a) ? b : a; }
__device__ __forceinline__ double sel_max(double a, double b) { return (b > a) ? b : a; }
__device__ __forceinline__ bool sign_clear(double v) { return __double2hiint(v) >= 0; }

// Nonzero after a bounded wait in a kernel gave up (read and cleared by take_device_status).
__device__ int g_vx_status = 0;
// Polls of the first wait for a TMA copy before giving up (settable for tests).
constexpr uint32_t kWaitPolls = 1u << 22;
__device__ uint32_t g_vx_wait_polls = kWaitPolls;

// Waits for phase `parity` of the barrier for at most `limit` polls; on give-up records the
// failure in g_vx_status and waits (bounded again) for the copy in flight before returning.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  const uint32_t limit = g_vx_wait_polls;
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(&g_vx_status, 1);
  for (uint32_t it = 0; it < kWaitPolls; ++it)  // the copy in flight must land before exit
    if (mbar_try_wait(bar, parity)) break;
  return false;
}

// C0 for one relation of a system of equations and inequalities: the enclosure [lo, hi]
// proves the relation false on the whole box (a NaN end proves nothing).
__device__ __forceinline__ bool rel_drops(double lo, double hi, int rel) {
  switch (rel) {
    case VX_LE: return lo > 0.0;
    case VX_GE: return hi < 0.0;
    case VX_LT: return lo >= 0.0;
    case VX_GT: return hi <= 0.0;
    default: return lo > 0.0 || hi < 0.0;
  }
}

// ---------------------------------------------------------------------------------------
// binary64 intervals
// ---------------------------------------------------------------------------------------
struct A64 {
  using V = double2;  // .x = lo, .y = hi
  struct X {
    double l, h;
    int cls;  // 1: X >= 0, -1: X <= 0, 0: X straddles 0
  };
  static __device__ __forceinline__ X box(const AxisGrid &g, int32_t t) {
    X x;
    endpoints(g, t, x.l, x.h);
    x.cls = (x.l >= 0.0) ? 1 : ((x.h <= 0.0) ? -1 : 0);
    return x;
  }
  template <int CLS>
  static __device__ __forceinline__ V step(V J, const X &x, V A) {
    double lo, hi;
    if (CLS > 0) {
      lo = __dmul_rd(J.x, sign_clear(J.x) ? x.l : x.h);
      hi = __dmul_ru(J.y, sign_clear(J.y) ? x.h : x.l);
    } else if (CLS < 0) {
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
  // 0: excluded, 1: kept (C0 of Sec. 3.2: excluded iff the enclosure proves the relation
  // false on the box; for an equation, iff 0 is provably outside)
  static __device__ __forceinline__ int classify(V J, int rel) {
    return rel_drops(J.x, J.y, rel) ? 0 : 1;
  }
  static __device__ __forceinline__ double lo(V J) { return J.x; }
  static __device__ __forceinline__ double hi(V J) { return J.y; }
  static __device__ __forceinline__ bool tight(V, float) { return false; }
  static __host__ __device__ __forceinline__ const V *coef(const PolyDev &p) { return p.c64; }
  static __host__ __device__ __forceinline__ const V *coef_fm(const PolyDev &p) { return p.c64_fm; }
};

// ---------------------------------------------------------------------------------------
// binary32 midpoint-radius
// ---------------------------------------------------------------------------------------
constexpr float kU32 = 0x1p-24f;    // unit roundoff of binary32
constexpr float kEta32 = 0x1p-149f;  // smallest positive binary32

struct A32 {
  using V = float2;  // .x = m, .y = r
  struct X {
    float m, r, a;  // a >= |m| + r
    float far;      // the end of largest magnitude, exactly (sign-definite boxes), else m
    bool split;     // far is exact and the box does not straddle 0
    int cls;
  };
  static __device__ __forceinline__ X box(const AxisGrid &g, int32_t t) {
    X x;
    if (g.fexact) {
      // every half-grid point is a binary32: centre and half-width are exact
      x.m = __fmaf_rn((float)t + 0.5f, g.fw, g.flo);
      x.r = 0.5f * g.fw;
    } else {
      double l, h;
      endpoints(g, t, l, h);
      x.m = __double2float_rn(0.5 * l + 0.5 * h);
      double dm = (double)x.m;
      x.r = __double2float_ru(fmax(__dadd_ru(h, -dm), __dadd_ru(dm, -l)));
    }
    x.a = __fadd_ru(fabsf(x.m), x.r);
    // on binary32-exact grids m +- r are the box's ends exactly
    x.split = g.fexact && !g.point && (x.m - x.r >= 0.f || x.m + x.r <= 0.f);
    x.far = x.split ? (x.m >= 0.f ? x.m + x.r : x.m - x.r) : x.m;
    x.cls = 0;  // one code path for every sign
    return x;
  }
  // On a box that does not straddle 0 the step uses the exact hull of J*X instead of the
  // general midpoint-radius product (whose interval exceeds the hull by 2 |Jm| Xr when J
  // straddles 0, and by 2 Jr Xr at one end otherwise, which matters on boxes near 0, where Xr
  // is comparable to |Xm|):
  //   J straddles 0 (|Jm| <= Jr): both ends of J*X at f, the end of X of largest magnitude:
  //     mid Jm f, radius Jr |f|;
  //   else, s = sign(Jm) sign(Xm): mid Jm Xm + s Jr Xr, radius |Jm| Xr + Jr |Xm|.
  // Rounding: t = RN(s Jr Xr + Am) and m = RN(Jm X' + t) each err by at most 2^-24 of their
  // result (2^-149 below the normal range, which the stored radius carries), both added to the
  // radius, rounded upward.  Other boxes take the general form.
  template <int CLS>
  static __device__ __forceinline__ V step(V J, const X &x, V A) {
    if (x.split) {
      const bool st = fabsf(J.x) <= J.y;
      const float sjr = (J.x >= 0.f) == (x.m >= 0.f) ? J.y : -J.y;
      const float t = __fmaf_rn(st ? 0.f : sjr, x.r, A.x);
      const float m = __fmaf_rn(J.x, st ? x.far : x.m, t);
      float r = __fmaf_ru(J.y, st ? x.a : fabsf(x.m), A.y);
      r = __fmaf_ru(st ? 0.f : fabsf(J.x), x.r, r);
      r = __fmaf_ru(kU32, fabsf(t), r);
      r = __fmaf_ru(kU32, fabsf(m), r);
      return make_float2(m, r);
    }
    float m = __fmaf_rn(J.x, x.m, A.x);
    float r = __fmaf_ru(J.y, x.a, A.y);
    r = __fmaf_ru(fabsf(J.x), x.r, r);
    r = __fmaf_ru(kU32, fabsf(m), r);
    return make_float2(m, r);
  }
  static __device__ __forceinline__ V store(V J) { return make_float2(J.x, __fadd_ru(J.y, kEta32)); }
  static __device__ __forceinline__ int classify(V J, int rel) {
    if (rel == VX_EQ) return (fabsf(J.x) > J.y) ? 0 : 1;
    return rel_drops(lo(J), hi(J), rel) ? 0 : 1;  // [m - r, m + r] rounded outward
  }
  static __device__ __forceinline__ double lo(V J) { return __dadd_rd((double)J.x, -(double)J.y); }
  static __device__ __forceinline__ double hi(V J) { return __dadd_ru((double)J.x, (double)J.y); }
  static __device__ __forceinline__ bool tight(V J, float theta) { return fabsf(J.x) >= theta * J.y; }
  static __host__ __device__ __forceinline__ const V *coef(const PolyDev &p) { return p.c32; }
  static __host__ __device__ __forceinline__ const V *coef_fm(const PolyDev &p) { return p.c32_fm; }
};

// ---------------------------------------------------------------------------------------
// binary32 intervals (lo, -hi) with an error bound certifying the binary64 decision
// ---------------------------------------------------------------------------------------
constexpr float kEta148 = 0x1p-148f;
constexpr float kCr = 0x1.000004p-24f;  // 2^-24 + 2^-46
constexpr float k2m27 = 0x1p-27f;
constexpr float k2m40 = 0x1p-40f;

struct A32C {
  using V = float4;  // .x = lo, .y = -hi, .z = E, .w unused
  struct X {
    float l, h, nl, nh;  // endpoints and their negations
    float xmaxp;         // >= xmax (1 + 2^-27)
    float cx;            // 2^-23 xmax when the endpoints are rounded outward, else 0
    int cls;
  };
  static __device__ __forceinline__ X box(const AxisGrid &g, int32_t t) {
    X x;
    x.cx = 0.f;
    if (g.fexact) {  // every half-grid point is a binary32 number: all exact
      if (g.point) {
        const float u = g.point == 1 ? 0.5f : (g.point == 3 ? 1.0f : 0.0f);
        x.l = x.h = __fmaf_rn((float)t + u, g.fw, g.flo);
      } else {
        x.l = __fmaf_rn((float)t, g.fw, g.flo);
        x.h = __fmaf_rn((float)t + 1.0f, g.fw, g.flo);
      }
    } else {
      double l, h;
      endpoints(g, t, l, h);
      x.l = __double2float_rd(l);
      x.h = __double2float_ru(h);
    }
    x.nl = -x.l;
    x.nh = -x.h;
    const float xm = fmaxf(fabsf(x.l), fabsf(x.h));
    x.xmaxp = __fmaf_ru(xm, k2m27, xm);
    if (!g.fexact) x.cx = __fmul_ru(xm, 0x1p-23f);
    // rounded endpoints take the sign-agnostic path, which carries the term c_x m_J
    x.cls = !g.fexact ? 0 : ((x.l >= 0.f) ? 1 : ((x.h <= 0.f) ? -1 : 0));
    return x;
  }
  // Both ends of J*X + A, each the min of two paired FMAs rounded to nearest: for X >= 0 the
  // lower end of J*X is min(lo_J l, lo_J h) and -hi is min(-hi_J l, -hi_J h); for X <= 0 the
  // roles of lo_J and -hi_J swap and the endpoints are negated.  No sign test on J: the two
  // chains (lo, -hi) never mix.
  template <int CLS>
  static __device__ __forceinline__ V step(V J, const X &x, V A) {
    float2 r;
    if (CLS != 0) {
      const float2 j = CLS > 0 ? make_float2(J.x, J.y) : make_float2(J.y, J.x);
      const float a = CLS > 0 ? x.l : x.nh, b = CLS > 0 ? x.h : x.nl;
      const float2 P = __ffma2_rn(j, make_float2(a, a), make_float2(A.x, A.y));
      const float2 Q = __ffma2_rn(j, make_float2(b, b), make_float2(A.x, A.y));
      r = make_float2(fminf(P.x, Q.x), fminf(P.y, Q.y));
    } else {  // X straddles 0: hull of the four products, each bound rounded once
      const float jh = -J.y;
      r.x = fminf(fminf(__fmaf_rn(J.x, x.l, A.x), __fmaf_rn(J.x, x.h, A.x)),
                  fminf(__fmaf_rn(jh, x.l, A.x), __fmaf_rn(jh, x.h, A.x)));
      r.y = fminf(fminf(__fmaf_rn(J.x, x.nl, A.y), __fmaf_rn(J.x, x.nh, A.y)),
                  fminf(__fmaf_rn(jh, x.nl, A.y), __fmaf_rn(jh, x.nh, A.y)));
    }
    const float m = fmaxf(fabsf(r.x), fabsf(r.y));
    float e = __fmaf_ru(kCr, m, A.z);
    if (CLS == 0) e = __fmaf_ru(fmaxf(fabsf(J.x), fabsf(J.y)), x.cx, e);
    e = __fmaf_ru(J.z, x.xmaxp, e);
    return make_float4(r.x, r.y, e, 0.f);
  }
  // a stored bound carries a relative margin 2^-40 and an absolute 2^-148
  static __device__ __forceinline__ V store(V J) {
    const float e = __fadd_ru(__fmaf_ru(J.z, k2m40, J.z), kEta148);
    return make_float4(J.x, J.y, e, e);  // the bound twice: a register pair for paired steps
  }
  // 0: the binary64 path surely excludes, 1: surely keeps, 2: inside the error band.  With
  // |lo32 - lo64| <= E and |hi32 - hi64| <= E: lo64 > 0 is sure when lo32 > E, lo64 <= 0 when
  // lo32 <= -E, lo64 >= 0 when lo32 >= E, lo64 < 0 when lo32 < -E (the same for hi, whose
  // negation J.y is stored).
  static __device__ __forceinline__ int classify(V J, int rel) {
    const bool fin = J.z < INFINITY;
    switch (rel) {
      case VX_LE:  // drop iff lo64 > 0
        return J.x > J.z ? 0 : ((J.x <= -J.z && fin) ? 1 : 2);
      case VX_GE:  // drop iff hi64 < 0
        return J.y > J.z ? 0 : ((J.y <= -J.z && fin) ? 1 : 2);
      case VX_LT:  // drop iff lo64 >= 0
        return J.x >= J.z ? 0 : ((J.x < -J.z && fin) ? 1 : 2);
      case VX_GT:  // drop iff hi64 <= 0
        return J.y >= J.z ? 0 : ((J.y < -J.z && fin) ? 1 : 2);
      default:
        if (J.x > J.z || J.y > J.z) return 0;                   // lo > E or hi < -E
        if (J.x <= -J.z && J.y <= -J.z && fin) return 1;       // lo <= -E, hi >= E, E finite
        return 2;
    }
  }
  static __device__ __forceinline__ double lo(V J) { return (double)J.x; }
  static __device__ __forceinline__ double hi(V J) { return -(double)J.y; }
  static __device__ __forceinline__ bool tight(V, float) { return false; }
  static __host__ __device__ __forceinline__ const V *coef(const PolyDev &p) { return p.c32c; }
  static __host__ __device__ __forceinline__ const V *coef_fm(const PolyDev &p) { return p.c32c_fm; }
};

// Algorithm 1 on one fibre: entries rowoff[a] + f (a = L-1 .. 0) of a block whose entry e is
// at base[e * stride].
template <class AR, int CLS>
__device__ __forceinline__ typename AR::V horner(const typename AR::V *__restrict__ base,
                                                 int64_t stride, const int32_t *rowoff, int f,
                                                 int L, const typename AR::X &x) {
  typename AR::V J = base[(int64_t)(rowoff[L - 1] + f) * stride];
#pragma unroll 4
  for (int a = L - 2; a >= 0; --a)
    J = AR::template step<CLS>(J, x, base[(int64_t)(rowoff[a] + f) * stride]);
  return J;
}

template <class AR>
__device__ __forceinline__ typename AR::V horner_any(const typename AR::V *__restrict__ base,
                                                     int64_t stride, const int32_t *rowoff,
                                                     int f, int L, const typename AR::X &x) {
  if (x.cls > 0) return horner<AR, 1>(base, stride, rowoff, f, L, x);
  if (x.cls < 0) return horner<AR, -1>(base, stride, rowoff, f, L, x);
  return horner<AR, 0>(base, stride, rowoff, f, L, x);
}

// the same for a single-fibre stage (entry a of the fibre is entry a of the block)
template <class AR, int CLS>
__device__ __forceinline__ typename AR::V horner1(const typename AR::V *__restrict__ base,
                                                  int64_t stride, int L, const typename AR::X &x) {
  typename AR::V J = base[(int64_t)(L - 1) * stride];
#pragma unroll 4
  for (int a = L - 2; a >= 0; --a) J = AR::template step<CLS>(J, x, base[(int64_t)a * stride]);
  return J;
}

// two fibres of the same length in lock-step (two independent chains per thread)
template <class AR, int CLS>
__device__ __forceinline__ void horner1x2(const typename AR::V *__restrict__ b0,
                                          const typename AR::V *__restrict__ b1, int L,
                                          const typename AR::X &x, typename AR::V &J0,
                                          typename AR::V &J1) {
  J0 = b0[L - 1];
  J1 = b1[L - 1];
#pragma unroll 2
  for (int a = L - 2; a >= 0; --a) {
    const typename AR::V A0 = b0[a], A1 = b1[a];
    J0 = AR::template step<CLS>(J0, x, A0);
    J1 = AR::template step<CLS>(J1, x, A1);
  }
}

template <class AR>
__device__ __forceinline__ void horner1x2_any(const typename AR::V *__restrict__ b0,
                                              const typename AR::V *__restrict__ b1, int L,
                                              const typename AR::X &x, typename AR::V &J0,
                                              typename AR::V &J1) {
  if (x.cls > 0)
    horner1x2<AR, 1>(b0, b1, L, x, J0, J1);
  else if (x.cls < 0)
    horner1x2<AR, -1>(b0, b1, L, x, J0, J1);
  else
    horner1x2<AR, 0>(b0, b1, L, x, J0, J1);
}

template <class AR>
__device__ __forceinline__ typename AR::V horner1_any(const typename AR::V *__restrict__ base,
                                                      int64_t stride, int L,
                                                      const typename AR::X &x) {
  if (x.cls > 0) return horner1<AR, 1>(base, stride, L, x);
  if (x.cls < 0) return horner1<AR, -1>(base, stride, L, x);
  return horner1<AR, 0>(base, stride, L, x);
}

// A block entry of the leaf stage rewritten for the summed bound: entry b (row b of the
// polynomial's single fibre, length L) keeps its binary32 ends and gets, in place of its bound
// E, B_b = RU((1 + 2^-50) E + kappa w_b M_b) + 2^-148, M_b = max(|lo|, |hi|) of the entry,
// w_b = min(b + 1, L - 1), kappa = 2^-24 (1 + 2^-23).  A leaf pair on y = |x| in
// [yl, yh] then bounds its distance to binary64 by e = Horner of B at xb = RU(yh (1 + 2^-23)),
// each step RU(e xb + B_b), instead of carrying the bound step by step from the magnitudes of
// its own partial values.  Why this bounds D = |lo32 - lo*| + |lo64 - lo*| (lo* exact): one
// step of a chain (value s, coefficient c, T = |s_prev| yh + |c|) gives
//   D <= (1 + 2^-50)(D_prev yh + E) + (2^-24 + 2^-50) T + 2^-149
// (binary32 rounds once to nearest, < 2^-24 T; binary64 rounds product and sum downward,
// < 2^-52 each of magnitudes <= T + D_prev yh + E), and |s| <= (1 + 2^-24) T + 2^-150, so
// T_a <= sum_{b >= a} M_b ((1 + 2^-24) yh)^(b - a); summing the recursion over the steps
// counts M_b once for each of the w_b steps a <= b, and every factor (1 + 2^-50)(1 + 2^-24)
// per power of yh is inside xb.  B_b >= E_b, so a per-step consumer of the block (A32C::step)
// stays sound on the rewritten entries.
__device__ __forceinline__ float4 bform_entry(const float4 v, int r, int L) {
  constexpr float kKappaB = 0x1.000002p-24f;  // >= 2^-24 + 2^-50
  const int w = r + 1 < L - 1 ? r + 1 : (L > 1 ? L - 1 : 0);
  const float M = fmaxf(fabsf(v.x), fabsf(v.y));
  float B = __fmaf_ru(__fmul_ru(kKappaB, (float)w), M, v.z);
  B = __fmaf_ru(v.z, 0x1p-50f, B);
  B = __fadd_ru(B, kEta148);
  return make_float4(v.x, v.y, B, B);
}

// A stage's output entry as stored: bfL > 0 (certified binary32, the last inner stage, whose
// blocks only the leaves read) rewrites it for the leaves' summed bound, row = its row in the
// leaf block (one fibre of bfL entries): the leaves then need no rewriting pass of their own.
template <class AR>
__device__ __forceinline__ typename AR::V out_entry(const typename AR::V &J, int bfL, int row) {
  if constexpr (std::is_same<AR, A32C>::value) {
    const float4 v = A32C::store(J);
    return bfL ? bform_entry(v, row, bfL) : v;
  } else {
    return AR::store(J);
  }
}

// Stage d < k-1 on every depth-d node.  Warp w takes node chunk w % nchunk (32 nodes, one per
// lane) and fibres g, g+G, ... with g = w / nchunk.  in: entry e of parent p's block at
// in[e * in_estride + p * in_nstride] (the coefficient tensor: in_estride 1, in_nstride 0).
// out: entry e of node i at out[e * out_estride + i * out_nstride]: entry-major
// (out_estride = nnodes, out_nstride = 1) when an inner stage reads it, node-major
// (out_estride = 1, out_nstride = blk_out) when the leaves do, so that a leaf's Horner walks
// consecutive entries of its parent's block.
// One warp's share of k_stage: nodes chunk*32 + lane (of nnodes), fibres g, g+G, ....  par
// holds parent indices of the parent array; poff is subtracted to index `in` (0 for one tree).
// FM: the parents' blocks are fibre-major (fibre f's entries at fiboff[f] .. fiboff[f]+L-1,
// consecutive, in_estride 1) instead of indexed through rowoff.
template <class AR, bool FM = false>
__device__ __forceinline__ void stage_chunk(const StageDev &st, const int32_t *outpos,
                                            const int32_t *rowoff,
                                            const int32_t *__restrict__ lab,
                                            const int32_t *__restrict__ par, int64_t poff,
                                            const typename AR::V *__restrict__ in,
                                            int64_t in_estride, int64_t in_nstride,
                                            typename AR::V *__restrict__ out, int64_t out_estride,
                                            int64_t out_nstride, int64_t nnodes, int64_t chunk,
                                            int grp, int G, const AxisGrid &g, int bfL = 0) {
  using V = typename AR::V;
  const int lane = threadIdx.x & 31;
  const int64_t node = chunk * 32 + lane;
  const bool live = node < nnodes;
  const int64_t nd = live ? node : nnodes - 1;  // idle lanes follow the last node, no store
  const V *base = par ? in + ((int64_t)__ldg(par + nd) - poff) * in_nstride : in;
  const typename AR::X x = AR::box(g, __ldg(lab + nd));
  V *dst = out + node * out_nstride;
  for (int f = grp; f < st.nfib; f += G) {
    const int L = __ldg(st.fiblen + f);
    const V J = FM ? horner1_any<AR>(base + __ldg(st.fiboff + f), 1, L, x)
                   : horner_any<AR>(base, in_estride, rowoff, f, L, x);
    const int o = __ldg(outpos + f);
    if (live) dst[(int64_t)o * out_estride] = out_entry<AR>(J, bfL, o);
  }
}

// Stage d < k-1 on every depth-d node.  Warp w takes node chunk w % nchunk (32 nodes, one per
// lane) and fibres g, g+G, ... with g = w / nchunk.  in: entry e of parent p's block at
// in[e * in_estride + p * in_nstride] (the coefficient tensor: in_estride 1, in_nstride 0).
// out: entry e of node i at out[e * out_estride + i * out_nstride]: entry-major
// (out_estride = nnodes, out_nstride = 1) when an inner stage reads it, node-major
// (out_estride = 1, out_nstride = blk_out) when the leaves do, so that a leaf's Horner walks
// consecutive entries of its parent's block.
template <class AR, bool FM = false>
__global__ void __launch_bounds__(kThreads)
    k_stage(const StageDev st, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
            const typename AR::V *__restrict__ in, int64_t in_estride, int64_t in_nstride,
            typename AR::V *__restrict__ out, int64_t out_estride, int64_t out_nstride,
            int64_t nnodes, int64_t nchunk, int G, AxisGrid g, int bfL) {
  extern __shared__ int32_t s_rowoff[];
  for (int i = threadIdx.x; i <= st.maxlen; i += blockDim.x) s_rowoff[i] = st.rowoff[i];
  __syncthreads();
  const int64_t nwarps = nchunk * G;
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); w < nwarps;
       w += (int64_t)gridDim.x * kWarpsPerBlock)
    stage_chunk<AR, FM>(st, st.outpos, s_rowoff, lab, par, 0, in, in_estride, in_nstride, out,
                        out_estride, out_nstride, nnodes, w % nchunk, (int)(w / nchunk), G, g,
                        bfL);
}

// Stage d (1 <= d < k-1) with the parent's block in shared memory.  The block is fibre-major
// (StageDev::fiboff), and CTA b takes parent p = b / G and the fibres of group g = b % G, a
// run of consecutive fibres holding about 1/G of the block's entries (stage_group), for all of
// p's children (the CSF child range ptr[p] .. ptr[p+1]-1, blockDim at a time, one child per
// thread).  The group's entries are one contiguous range, brought in by a TMA bulk copy
// (cp.async.bulk, completion on an mbarrier), so a CTA holds only its share of the block; every
// Horner step then reads consecutive shared-memory entries at an address common to the whole
// CTA (a broadcast).
//
// The fibres [fb, fe) of group g of G: those whose first entry lies in [g T / G, (g+1) T / G)
// (T = blk_in; fibres are not split), and the entry range [c_lo, c_hi) to copy: [fiboff[fb],
// fiboff[fe]) widened to 16-byte boundaries (entries of 8 bytes pair up; blk_in is even then).
struct StageGroup {
  int fb, fe;
  int64_t c_lo, c_hi;
};

__device__ __forceinline__ int fibre_at_or_after(const int32_t *__restrict__ fiboff, int nfib,
                                                 int64_t e) {
  int lo = 0, hi = nfib;  // the first fibre f with fiboff[f] >= e (nfib if none)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(fiboff + mid) < e) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

template <int ESZ>
__device__ __forceinline__ StageGroup stage_group(const StageDev &st, int grp, int G) {
  StageGroup r;
  r.fb = fibre_at_or_after(st.fiboff, st.nfib, (int64_t)grp * st.blk_in / G);
  r.fe = grp + 1 == G ? st.nfib : fibre_at_or_after(st.fiboff, st.nfib, (int64_t)(grp + 1) * st.blk_in / G);
  constexpr int per = 16 / ESZ;  // entries per 16 bytes
  r.c_lo = (int64_t)__ldg(st.fiboff + r.fb) / per * per;
  r.c_hi = ((int64_t)__ldg(st.fiboff + r.fe) + per - 1) / per * per;
  return r;
}

// One thread: the bulk copy of entries [c_lo, c_hi) of parent p's block into s_blk.
template <class V>
__device__ __forceinline__ void stage_group_copy(const V *in, int64_t p, int64_t blk,
                                                 const StageGroup &r, uint64_t *bar, V *s_blk) {
  mbar_init(bar, 1);
  const uint64_t bytes = (uint64_t)(r.c_hi - r.c_lo) * sizeof(V);
  mbar_arrive_expect_tx(bar, (uint32_t)bytes);
  const char *src = reinterpret_cast<const char *>(in + p * blk + r.c_lo);
  char *dst = reinterpret_cast<char *>(s_blk);
  for (uint64_t o = 0; o < bytes; o += 32768) {
    const uint32_t n = (uint32_t)(bytes - o < 32768 ? bytes - o : 32768);
    bulk_copy_g2s(dst + o, src + o, n, bar);
  }
}

template <class AR>
__global__ void __launch_bounds__(512)
    k_stage_tma(const StageDev st, const int32_t *__restrict__ lab,
                const int32_t *__restrict__ pptr, const typename AR::V *__restrict__ in,
                typename AR::V *__restrict__ out, int64_t out_estride, int64_t out_nstride,
                int G, AxisGrid g, int bfL) {
  using V = typename AR::V;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  V *s_blk = reinterpret_cast<V *>(smem + 128);
  const int64_t p = blockIdx.x / G;
  const StageGroup r = stage_group<(int)sizeof(V)>(st, (int)(blockIdx.x % G), G);
  if (r.fb >= r.fe) return;  // an empty group (the same for the whole CTA)
  const int64_t c0 = __ldg(pptr + p), c1 = __ldg(pptr + p + 1);
  if (threadIdx.x == 0) stage_group_copy(in, p, st.blk_in, r, bar, s_blk);
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0)) return;
  for (int64_t n0 = c0; n0 < c1; n0 += blockDim.x) {
    const int64_t node = n0 + threadIdx.x;
    const bool live = node < c1;
    const int64_t nd = live ? node : c1 - 1;
    const typename AR::X x = AR::box(g, __ldg(lab + nd));
    V *dst = out + node * out_nstride;
    for (int f = r.fb; f < r.fe; ++f) {
      const int L = __ldg(st.fiblen + f);
      const V J = horner1_any<AR>(s_blk + (__ldg(st.fiboff + f) - r.c_lo), 1, L, x);
      const int o = __ldg(st.outpos + f);
      if (live) dst[(int64_t)o * out_estride] = out_entry<AR>(J, bfL, o);
    }
  }
}

struct LeafArgs {
  const void *in[VX_MAXPOLY];  // parent blocks per polynomial, node-major (the coefficients
                               // when k == 1)
  int64_t blk[VX_MAXPOLY];     // entries per parent block (0 when k == 1)
  int32_t len[VX_MAXPOLY];
  int8_t rel[VX_MAXPOLY];      // VX_EQ .. VX_GT per polynomial
};

// Last stage on leaf i: one Horner per polynomial, then C0 (par: parent indices, minus poff
// to index the blocks of A).
template <class AR>
__device__ __forceinline__ void leaf_item(const LeafArgs &A, int npoly,
                                          const int32_t *__restrict__ lab,
                                          const int32_t *__restrict__ par, int64_t poff,
                                          int64_t i, int64_t nleaves, const AxisGrid &g,
                                          uint8_t *__restrict__ keep, double *__restrict__ lo,
                                          double *__restrict__ hi, uint8_t *__restrict__ flag,
                                          float theta) {
  using V = typename AR::V;
  const typename AR::X x = AR::box(g, __ldg(lab + i));
  const int64_t p = par ? (int64_t)__ldg(par + i) - poff : 0;
  bool excl = false, amb = false, tg = false;
  auto decide = [&](int f, const V &J) {
    if (lo) {
      lo[(int64_t)f * nleaves + i] = AR::lo(J);
      hi[(int64_t)f * nleaves + i] = AR::hi(J);
    }
    const int c = AR::classify(J, A.rel[f]);
    excl = excl || c == 0;
    amb = amb || c == 2;
    tg = tg || AR::tight(J, theta);
  };
  int f = 0;
  for (; f + 1 < npoly && A.len[f] == A.len[f + 1]; f += 2) {
    V J0, J1;
    horner1x2_any<AR>((const V *)A.in[f] + p * A.blk[f], (const V *)A.in[f + 1] + p * A.blk[f + 1],
                      A.len[f], x, J0, J1);
    decide(f, J0);
    decide(f + 1, J1);
  }
  for (; f < npoly; ++f) {
    const V *base = (const V *)A.in[f] + p * A.blk[f];
    decide(f, horner1_any<AR>(base, 1, A.len[f], x));
  }
  keep[i] = excl ? 0 : 1;
  if (flag) flag[i] = (!excl && (amb || tg)) ? 1 : 0;
}

// Last stage on every leaf: one Horner per polynomial, then C0.  Lane = leaf.
template <class AR>
__global__ void __launch_bounds__(kThreads)
    k_leaf(LeafArgs A, int npoly, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
           int64_t nleaves, AxisGrid g, uint8_t *__restrict__ keep, double *__restrict__ lo,
           double *__restrict__ hi, uint8_t *__restrict__ flag, float theta) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += stride)
    leaf_item<AR>(A, npoly, lab, par, 0, i, nleaves, g, keep, lo, hi, flag, theta);
}

// Last stage in the certified binary32 arithmetic, two consecutive leaves per thread.  When
// every thread of a warp holds two leaves of one parent whose x_k intervals do not straddle 0
// (always so at level >= 1 of a grid exact in binary32), the two leaves share every
// coefficient load, and a leaf with x_k <= 0 runs Horner in y = -x_k (step_y2), so the
// lanes of the warp run the same instructions whatever the signs of their boxes.  Any other
// warp takes the per-leaf path of k_leaf.
struct YLeaf {
  float yl, yh, xmaxp;
  float xb;  // RU(yh (1 + 2^-23)): the multiplier of the summed bound (bform_entry)
  bool neg;
};

__device__ __forceinline__ YLeaf yleaf(const A32C::X &x) {
  YLeaf y;
  y.neg = x.cls < 0;
  y.yl = y.neg ? x.nh : x.l;
  y.yh = y.neg ? x.nl : x.h;
  y.xmaxp = x.xmaxp;
  y.xb = __fmaf_ru(y.yh, 0x1p-23f, y.yh);
  return y;
}

__device__ __forceinline__ float4 negated(float4 A) { return make_float4(A.y, A.x, A.z, A.w); }

// Two leaves (or nodes) of one parent stepped together: per leaf the pair (lo, -hi) of its
// chain, and the two error bounds as one pair, so that the bound's two FMAs per step serve
// both leaves as paired instructions (a stored entry carries its bound twice, in .z and .w).
struct YPair {
  float2 l0, h0, l1, h1;  // (yl, yl) and (yh, yh) of leaf 0 and leaf 1
  float2 xm;              // (xmaxp of leaf 0, xmaxp of leaf 1)
  float xb;               // max(xb of leaf 0, xb of leaf 1): the pair's summed-bound multiplier
  bool neg0, neg1;
};

__device__ __forceinline__ YPair ypair(const YLeaf &a, const YLeaf &b) {
  YPair y;
  y.l0 = make_float2(a.yl, a.yl);
  y.h0 = make_float2(a.yh, a.yh);
  y.l1 = make_float2(b.yl, b.yl);
  y.h1 = make_float2(b.yh, b.yh);
  y.xm = make_float2(a.xmaxp, b.xmaxp);
  y.xb = fmaxf(a.xb, b.xb);
  y.neg0 = a.neg;
  y.neg1 = b.neg;
  return y;
}

// One step of A32C on y = |x| >= 0, y = [yl, yh], for both leaves: Horner in x <= 0 is Horner
// in y = -x on the coefficients (-1)^a A_a, the state being (-1)^a J_a (exact: interval
// negation swaps the pair (lo, -hi), and the products are the same reals).  SW = 0 takes the
// entry as it is, 1 negated for both leaves (a pair swap), 2 negated per leaf where sw0 / sw1.
// OSW: the chains hold -J (the pair (-hi, lo)), so that J_a = (-J_{a+1}) y + A_a takes every
// entry as it is, and the step writes its two minima in swapped order (the same products and
// roundings as SW = 1 on the odd entries, without moving the entry's pair).
// Each end is the min of two paired FMAs rounded to nearest; the bounds follow A32C::step's
// recursion, both leaves' in one paired FMA pair.
// BF: the entry's .z/.w hold the summed bound B of bform_entry, and one bound serves both
// leaves: e = RU(e xb + B) with xb the larger of their multipliers (every term of the
// recursion is >= 0 and RU is monotone, so it bounds each leaf's own recursion), one FMA per
// step and no magnitude of the step's result.  The bound lives in e.x (e.y is not used).
template <int SW, bool BF = false, bool OSW = false>
__device__ __forceinline__ void step_y2(float2 &j0, float2 &j1, float2 &e, const YPair &y,
                                        const float4 &A, bool sw0, bool sw1) {
  float2 c0, c1;
  if (SW == 0) {
    c0 = c1 = make_float2(A.x, A.y);
  } else if (SW == 1) {
    c0 = c1 = make_float2(A.y, A.x);
  } else {
    c0 = sw0 ? make_float2(A.y, A.x) : make_float2(A.x, A.y);
    c1 = sw1 ? make_float2(A.y, A.x) : make_float2(A.x, A.y);
  }
  const float2 P0 = __ffma2_rn(j0, y.l0, c0), Q0 = __ffma2_rn(j0, y.h0, c0);
  const float2 P1 = __ffma2_rn(j1, y.l1, c1), Q1 = __ffma2_rn(j1, y.h1, c1);
  if (OSW) {
    j0 = make_float2(fminf(P0.y, Q0.y), fminf(P0.x, Q0.x));
    j1 = make_float2(fminf(P1.y, Q1.y), fminf(P1.x, Q1.x));
  } else {
    j0 = make_float2(fminf(P0.x, Q0.x), fminf(P0.y, Q0.y));
    j1 = make_float2(fminf(P1.x, Q1.x), fminf(P1.y, Q1.y));
  }
  if (BF) {
    e.x = __fmaf_ru(e.x, y.xb, A.z);
  } else {
    const float2 m =
        make_float2(fmaxf(fabsf(j0.x), fabsf(j0.y)), fmaxf(fabsf(j1.x), fabsf(j1.y)));
    e = __ffma2_ru(e, y.xm, __ffma2_ru(make_float2(kCr, kCr), m, make_float2(A.z, A.w)));
  }
}

// SGN: +1 no leaf negated, -1 both negated (warp-uniform cases: SGN = -1 runs the chains as
// -J, OSW), 0 per leaf at run time (odd entries swapped per leaf).
template <int SGN>
struct SwapOdd {
  static constexpr int value = SGN == 0 ? 2 : 0;
  static constexpr bool osw = SGN < 0;
};

// The chain's first state from its top entry A_{L-1}: J (or -J under OSW), for each leaf.
template <int SGN>
__device__ __forceinline__ void top_state(const float4 &A, bool top_odd, const YPair &y,
                                          float2 &j0, float2 &j1) {
  if (SwapOdd<SGN>::osw) {
    j0 = j1 = make_float2(A.y, A.x);
  } else {
    const float4 A0 = (top_odd && y.neg0) ? negated(A) : A;
    const float4 A1 = (top_odd && y.neg1) ? negated(A) : A;
    j0 = make_float2(A0.x, A0.y);
    j1 = make_float2(A1.x, A1.y);
  }
}

// The chain's value at a = 0 as the entry (lo, -hi, bound, bound).
template <int SGN>
__device__ __forceinline__ float4 chain_out(const float2 &j, float e) {
  return SwapOdd<SGN>::osw ? make_float4(j.y, j.x, e, e) : make_float4(j.x, j.y, e, e);
}

// Horner of NP polynomials of one length L on the leaves of y (one parent): chain f of leaf c
// is (-1)^a J_a (equal to J_a when the leaf is not negated).  Odd entries are negated for a
// negated leaf; the loop takes the entries in (odd, even) pairs, loaded one pair ahead.
template <int NP, int SGN, bool BF = false>
__device__ __forceinline__ void horner_y2(const float4 *const (&b)[2], int L, const YPair &y,
                                          float4 (&K0)[2], float4 (&K1)[2]) {
  constexpr int SWO = SwapOdd<SGN>::value;
  constexpr bool OSW = SwapOdd<SGN>::osw;
  const bool top_odd = (L - 1) & 1;
  float2 j0[NP], j1[NP], e[NP];
#pragma unroll
  for (int f = 0; f < NP; ++f) {
    const float4 A = b[f][L - 1];
    top_state<SGN>(A, top_odd, y, j0[f], j1[f]);
    e[f] = make_float2(A.z, A.w);
  }
  int a = L - 2;
  if (a >= 0 && !(a & 1)) {
#pragma unroll
    for (int f = 0; f < NP; ++f)
      step_y2<0, BF, OSW>(j0[f], j1[f], e[f], y, b[f][a], false, false);
    --a;
  }
  // two (odd, even) pairs per trip: half the loop and address overhead per step; the entries
  // are walked by pointer (immediate offsets) with a trip counter
  if (a >= 3) {
    const float4 *pa[NP];
#pragma unroll
    for (int f = 0; f < NP; ++f) pa[f] = b[f] + a;
    int trips = (a + 1) >> 2;
    a -= 4 * trips;
    for (; trips > 0; --trips) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 A[NP], B[NP];
#pragma unroll
        for (int f = 0; f < NP; ++f) {
          A[f] = pa[f][-2 * h];
          B[f] = pa[f][-2 * h - 1];
        }
#pragma unroll
        for (int f = 0; f < NP; ++f) {
          step_y2<SWO, BF, OSW>(j0[f], j1[f], e[f], y, A[f], y.neg0, y.neg1);
          step_y2<0, BF, OSW>(j0[f], j1[f], e[f], y, B[f], false, false);
        }
      }
#pragma unroll
      for (int f = 0; f < NP; ++f) pa[f] -= 4;
    }
  }
  if (a >= 1) {
    float4 A[NP], B[NP];
#pragma unroll
    for (int f = 0; f < NP; ++f) {
      A[f] = b[f][a];
      B[f] = b[f][a - 1];
    }
#pragma unroll
    for (int f = 0; f < NP; ++f) {
      step_y2<SWO, BF, OSW>(j0[f], j1[f], e[f], y, A[f], y.neg0, y.neg1);
      step_y2<0, BF, OSW>(j0[f], j1[f], e[f], y, B[f], false, false);
    }
  }
#pragma unroll
  for (int f = 0; f < NP; ++f) {
    K0[f] = chain_out<SGN>(j0[f], e[f].x);
    K1[f] = chain_out<SGN>(j1[f], BF ? e[f].x : e[f].y);
  }
}

// Horner of fibre f of a block (entries rowoff[a] + f, a = L-1 .. 0; entry e at
// base[e * estride]) on two boxes of one parent, as horner_y2 does for a leaf's single fibre.
template <int SGN>
__device__ __forceinline__ void horner_y2_fibre(const float4 *__restrict__ base, int64_t estride,
                                                const int32_t *rowoff, int f, int L,
                                                const YPair &y, float4 &K0, float4 &K1) {
  constexpr int SWO = SwapOdd<SGN>::value;
  constexpr bool OSW = SwapOdd<SGN>::osw;
  auto ent = [&](int a) { return base[(int64_t)(rowoff[a] + f) * estride]; };
  const bool top_odd = (L - 1) & 1;
  float2 j0, j1, e;
  {
    const float4 A = ent(L - 1);
    top_state<SGN>(A, top_odd, y, j0, j1);
    e = make_float2(A.z, A.w);
  }
  int a = L - 2;
  if (a >= 0 && !(a & 1)) {
    step_y2<0, false, OSW>(j0, j1, e, y, ent(a), false, false);
    --a;
  }
  float4 An = make_float4(0.f, 0.f, 0.f, 0.f), Bn = An;
  if (a >= 1) {
    An = ent(a);
    Bn = ent(a - 1);
  }
  for (; a >= 1; a -= 2) {
    const float4 A = An, B = Bn;
    if (a >= 3) {
      An = ent(a - 2);
      Bn = ent(a - 3);
    }
    step_y2<SWO, false, OSW>(j0, j1, e, y, A, y.neg0, y.neg1);
    step_y2<0, false, OSW>(j0, j1, e, y, B, false, false);
  }
  K0 = chain_out<SGN>(j0, e.x);
  K1 = chain_out<SGN>(j1, e.y);
}

// The warp-uniform sign case of a leaf pair: +1 no lane negated, -1 all negated, 0 mixed.
__device__ __forceinline__ int warp_sign(const YPair &y) {
  if (__all_sync(0xffffffffu, !y.neg0 && !y.neg1)) return 1;
  if (__all_sync(0xffffffffu, y.neg0 && y.neg1)) return -1;
  return 0;
}

// ---------------------------------------------------------------------------------------
// Taylor form (Def. 3) at the leaves: the system holds G_a = d^a F / a! for the multi-indices
// |a| <= m of one polynomial F (lexicographic order); G_a with |a| < m was partially evaluated
// at the box centres (point grids), the others on the boxes.  Per leaf, with V_a the value of
// G_a and x - c in [-r, r]:
//   T = sum_a V_a * prod_i range((x_i - c_i)^{a_i}),
// the range [1,1] (a_i = 0), [0, r^a_i] (even) or [-r^a_i, r^a_i] (odd); interval products
// are hulls of directed endpoint products, sums outward, in the order of the multi-indices.
// C0 on T.  With c1 (m >= 2, one equation) also the inclusion criterion C1 of Sec. 3.2 on the
// Taylor form: s_i = +1 if the midpoint of g_i = V_{e_i} (a first derivative at the centre)
// is >= 0 (lo >= -hi), else -1; V_max = c + s r and V_min = c - s r are the vertices where
// the linear part is largest and smallest; F(V) lies in sum_a V_a prod_i [v_i, v_i]^{a_i}
// (v = V - c, powers by repeated interval products); certified iff that enclosure is > 0 at
// V_max and < 0 at V_min (opposite signs at two points of the connected box).
// ---------------------------------------------------------------------------------------
struct TaylorLeaf {
  int32_t na, m, k;
  int8_t alpha[VX_MAXPOLY][VX_KMAX];
  double r[VX_KMAX];  // half-widths of the level's boxes, per axis
  int32_t first;      // 1: write keep, 0: AND into it (several polynomials)
  double *lo, *hi;    // nullable: T per leaf
  int32_t rel;        // the polynomial's relation (VX_EQ .. VX_GT)
  int32_t c1;         // nonzero: write inc (C1 on the Taylor form)
  int8_t ei[VX_KMAX]; // index of the multi-index e_i
  uint8_t *inc;
  uint8_t *flag;      // certified binary32 only: 1 where a decision is left to binary64
};

__device__ __forceinline__ double2 imul_hull(double2 x, double2 y) {
  double2 r;
  r.x = sel_min(sel_min(__dmul_rd(x.x, y.x), __dmul_rd(x.x, y.y)),
                sel_min(__dmul_rd(x.y, y.x), __dmul_rd(x.y, y.y)));
  r.y = sel_max(sel_max(__dmul_ru(x.x, y.x), __dmul_ru(x.x, y.y)),
                sel_max(__dmul_ru(x.y, y.x), __dmul_ru(x.y, y.y)));
  return r;
}

__device__ __forceinline__ double2 pow_range(double r, int a) {
  if (a == 0) return make_double2(1.0, 1.0);
  double p = r;
  for (int i = 1; i < a; ++i) p = __dmul_ru(p, r);
  return make_double2((a & 1) ? -p : 0.0, p);
}

__global__ void __launch_bounds__(kThreads)
    k_leaf_taylor(LeafArgs A, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
                  int64_t nleaves, AxisGrid gbox, AxisGrid gpoint, TaylorLeaf T,
                  uint8_t *__restrict__ keep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += stride) {
    const int32_t t = __ldg(lab + i);
    const A64::X xb = A64::box(gbox, t), xp = A64::box(gpoint, t);
    const int64_t p = par ? (int64_t)__ldg(par + i) : 0;
    double2 V[VX_MAXPOLY];
    double2 acc = make_double2(0.0, 0.0);
    for (int a = 0; a < T.na; ++a) {
      int tot = 0;
      for (int d = 0; d < T.k; ++d) tot += T.alpha[a][d];
      const double2 *base = (const double2 *)A.in[a] + p * A.blk[a];
      V[a] = horner1_any<A64>(base, 1, A.len[a], tot < T.m ? xp : xb);
      double2 P = make_double2(1.0, 1.0);
      for (int d = 0; d < T.k; ++d) P = imul_hull(P, pow_range(T.r[d], T.alpha[a][d]));
      const double2 VP = imul_hull(V[a], P);
      acc = make_double2(__dadd_rd(acc.x, VP.x), __dadd_ru(acc.y, VP.y));
    }
    if (T.lo) {
      T.lo[i] = acc.x;
      T.hi[i] = acc.y;
    }
    const uint8_t k0 = rel_drops(acc.x, acc.y, T.rel) ? 0 : 1;
    keep[i] = T.first ? k0 : (uint8_t)(keep[i] & k0);
    if (T.c1) {
      double v[VX_KMAX];
      for (int d = 0; d < T.k; ++d) {
        const double2 g = V[T.ei[d]];
        v[d] = (g.x >= -g.y) ? T.r[d] : -T.r[d];
      }
      double2 at[2];
      for (int side = 0; side < 2; ++side) {  // 0: V_max, 1: V_min
        double2 sum = make_double2(0.0, 0.0);
        for (int a = 0; a < T.na; ++a) {
          double2 P = make_double2(1.0, 1.0);
          for (int d = 0; d < T.k; ++d) {
            const double x = side == 0 ? v[d] : -v[d];
            for (int e = 0; e < T.alpha[a][d]; ++e) P = imul_hull(P, make_double2(x, x));
          }
          const double2 VP = imul_hull(V[a], P);
          sum = make_double2(__dadd_rd(sum.x, VP.x), __dadd_ru(sum.y, VP.y));
        }
        at[side] = sum;
      }
      T.inc[i] = (at[0].x > 0.0 && at[1].y < 0.0) ? 1 : 0;
    }
  }
}

// The Taylor form in the certified binary32 arithmetic: each G_a's value V_a comes with the
// bound E_a on the distance of its ends to the binary64 ones.  The binary64 form T64 then lies
// in the form of the wide intervals [lo-E, hi+E], and T64.lo / T64.hi are bounded above /
// below through single points of the possible ends (U, L below), which works for thin (point)
// values too: C0 drops the box surely when the wide form proves the relation false, keeps it
// surely when the bounds show that T64 cannot be dropped; C1 (m >= 2) is sure when the signs
// of the gradient's midpoints are (|lo + hi| > 2E) and the same bounds at V_max, V_min decide
// it.  Every other box is flagged for the binary64 Taylor form.  keep (first = 1) or keep &=
// the sure-or-unsure keep; flag |= unsure.
__global__ void __launch_bounds__(kThreads)
    k_leaf_taylor_c(LeafArgs A, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
                    int64_t nleaves, AxisGrid gbox, AxisGrid gpoint, TaylorLeaf T,
                    uint8_t *__restrict__ keep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += stride) {
    const int32_t t = __ldg(lab + i);
    const A32C::X xb = A32C::box(gbox, t), xp = A32C::box(gpoint, t);
    const int64_t p = par ? (int64_t)__ldg(par + i) : 0;
    float4 V[VX_MAXPOLY];  // (lo, -hi, E) of every G_a
    bool finite = true;
    for (int a = 0; a < T.na; ++a) {
      int tot = 0;
      for (int d = 0; d < T.k; ++d) tot += T.alpha[a][d];
      const float4 *base = (const float4 *)A.in[a] + p * A.blk[a];
      V[a] = horner1_any<A32C>(base, 1, A.len[a], tot < T.m ? xp : xb);
      finite = finite && isfinite(V[a].x) && isfinite(V[a].y) && isfinite(V[a].z);
    }
    // G_a's binary64 value [l64, h64] has l64 in [lo-E, lo+E] and h64 in [hi-E, hi+E]: the
    // wide interval [lo-E, hi+E] contains it; and for any factor P, lo(V*P) <= l64 p for each
    // end p of P, so lo(V*P) <= min_p max(RU((lo-E) p), RU((lo+E) p)) =: U, and likewise
    // hi(V*P) >= max_p min(RD((hi-E) p), RD((hi+E) p)) =: L, even when V is thin (a point).
    auto ends = [&](int a, double &l1, double &l2, double &h1, double &h2) {
      const double e = (double)V[a].z, lo = (double)V[a].x, hi = -(double)V[a].y;
      l1 = __dadd_rd(lo, -e);
      l2 = __dadd_ru(lo, e);
      h1 = __dadd_rd(hi, -e);
      h2 = __dadd_ru(hi, e);
    };
    // one term V_a * P (P = [pl, ph]): its wide enclosure and the bounds U, L above
    auto term = [&](int a, double2 P, double2 &w, double &u, double &l) {
      double l1, l2, h1, h2;
      ends(a, l1, l2, h1, h2);
      w = imul_hull(make_double2(l1, h2), P);
      u = sel_min(sel_max(__dmul_ru(l1, P.x), __dmul_ru(l2, P.x)),
                  sel_max(__dmul_ru(l1, P.y), __dmul_ru(l2, P.y)));
      l = sel_max(sel_min(__dmul_rd(h1, P.x), __dmul_rd(h2, P.x)),
                  sel_min(__dmul_rd(h1, P.y), __dmul_rd(h2, P.y)));
    };
    // the form with the box's ranges (C0): T64 lies in tw, T64.lo <= tu, T64.hi >= tl
    double2 tw = make_double2(0.0, 0.0);
    double tu = 0.0, tlo = 0.0;
    for (int a = 0; a < T.na; ++a) {
      double2 P = make_double2(1.0, 1.0);
      for (int d = 0; d < T.k; ++d) P = imul_hull(P, pow_range(T.r[d], T.alpha[a][d]));
      double2 w;
      double u, l;
      term(a, P, w, u, l);
      tw = make_double2(__dadd_rd(tw.x, w.x), __dadd_ru(tw.y, w.y));
      tu = __dadd_ru(tu, u);
      tlo = __dadd_rd(tlo, l);
    }
    int c0 = 2;  // 0 sure exclusion, 1 sure keep, 2 unsure
    if (finite && rel_drops(tw.x, tw.y, T.rel)) c0 = 0;
    else if (finite && !rel_drops(tu, tlo, T.rel)) c0 = 1;  // some T64 between them keeps
    bool unsure = c0 == 2;
    if (T.c1) {
      // the vertex choice needs the sign of lo + hi of each first derivative, which is within
      // 2E of the binary32 sum
      double v[VX_KMAX];
      bool signs = finite;
      for (int d = 0; d < T.k; ++d) {
        const float4 g = V[T.ei[d]];
        const double e2 = __dmul_ru(2.0, (double)g.z);
        const double slo = __dadd_rd(__dadd_rd((double)g.x, -(double)g.y), -e2);
        const double shi = __dadd_ru(__dadd_ru((double)g.x, -(double)g.y), e2);
        const bool pos = slo >= 0.0, neg = shi < 0.0;
        signs = signs && (pos || neg);
        v[d] = pos ? T.r[d] : -T.r[d];
      }
      int inc = 2;  // 0 surely not certified, 1 surely certified, 2 unsure
      if (signs) {
        double2 aw[2];
        double au[2], al[2];
        for (int side = 0; side < 2; ++side) {  // 0: V_max, 1: V_min
          double2 sw = make_double2(0.0, 0.0);
          double su = 0.0, sl = 0.0;
          for (int a = 0; a < T.na; ++a) {
            double2 P = make_double2(1.0, 1.0);
            for (int d = 0; d < T.k; ++d) {
              const double x = side == 0 ? v[d] : -v[d];
              for (int e = 0; e < T.alpha[a][d]; ++e) P = imul_hull(P, make_double2(x, x));
            }
            double2 w;
            double u, l;
            term(a, P, w, u, l);
            sw = make_double2(__dadd_rd(sw.x, w.x), __dadd_ru(sw.y, w.y));
            su = __dadd_ru(su, u);
            sl = __dadd_rd(sl, l);
          }
          aw[side] = sw;
          au[side] = su;
          al[side] = sl;
        }
        // certified: lower end at V_max > 0 and upper end at V_min < 0
        if (aw[0].x > 0.0 && aw[1].y < 0.0) inc = 1;
        else if (au[0] <= 0.0 || al[1] >= 0.0) inc = 0;
      }
      unsure = unsure || (c0 != 0 && inc == 2);
      T.inc[i] = inc == 1 ? 1 : 0;
    }
    const uint8_t k0 = c0 == 0 ? 0 : 1;
    keep[i] = T.first ? k0 : (uint8_t)(keep[i] & k0);
    const uint8_t fl = unsure ? 1 : 0;
    T.flag[i] = T.first ? fl : (uint8_t)(T.flag[i] | fl);
  }
}

// Inclusion criterion C1 by vertex signs: after each vertex's evaluation (point intervals at
// one corner of every box), flags |= 1 if the value is certified > 0, |= 2 if < 0.
__global__ void k_c1_fold(const double *__restrict__ lo, const double *__restrict__ hi,
                          int64_t n, uint8_t *__restrict__ flags, int first) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint8_t f = (lo[i] > 0.0 ? 1 : 0) | (hi[i] < 0.0 ? 2 : 0);
    flags[i] = first ? f : (uint8_t)(flags[i] | f);
  }
}

__global__ void k_c1_final(const uint8_t *__restrict__ flags, int64_t n,
                           uint8_t *__restrict__ inc) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    inc[i] = flags[i] == 3 ? 1 : 0;
}

// One warp's share of k_stage_c: node pairs of chunk `chunk` (64 nodes), fibres g, g+G, ....
// A warp whose 32 pairs each share a parent and do not straddle 0 shares every load between
// the two nodes and runs sign-free (horner_y2_fibre); any other warp takes k_stage's per-node
// path.  par/poff and FM as in stage_chunk.
template <bool FM = false>
__device__ __forceinline__ void stage_chunk_c(const StageDev &st, const int32_t *outpos,
                                              const int32_t *rowoff,
                                              const int32_t *__restrict__ lab,
                                              const int32_t *__restrict__ par, int64_t poff,
                                              const float4 *__restrict__ in, int64_t in_estride,
                                              int64_t in_nstride, float4 *__restrict__ out,
                                              int64_t out_estride, int64_t out_nstride,
                                              int64_t nnodes, int64_t chunk, int grp, int G,
                                              const AxisGrid &g, int bfL = 0) {
  const int lane = threadIdx.x & 31;
  const int64_t npairs = (nnodes + 1) >> 1;
  const int64_t q = chunk * 32 + lane;
  const bool live = q < npairs;
  const int64_t i0 = 2 * (live ? q : npairs - 1);
  const bool two = live && i0 + 1 < nnodes;
  const int64_t i1 = i0 + 1 < nnodes ? i0 + 1 : i0;
  const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
  const int64_t p0 = par ? (int64_t)__ldg(par + i0) - poff : 0;
  const int64_t p1 = par ? (int64_t)__ldg(par + i1) - poff : 0;
  const bool fast = p0 == p1 && x0.cls != 0 && x1.cls != 0;
  if (__all_sync(0xffffffffu, fast)) {
    const YPair yp = ypair(yleaf(x0), yleaf(x1));
    const int ws = warp_sign(yp);
    const float4 *base = in + p0 * in_nstride;
    for (int f = grp; f < st.nfib; f += G) {
      const int L = __ldg(st.fiblen + f);
      float4 K0, K1;
      if (FM) {
        const float4 *const b[2] = {base + __ldg(st.fiboff + f), nullptr};
        float4 K0v[2], K1v[2];
        if (ws > 0)
          horner_y2<1, 1>(b, L, yp, K0v, K1v);
        else if (ws < 0)
          horner_y2<1, -1>(b, L, yp, K0v, K1v);
        else
          horner_y2<1, 0>(b, L, yp, K0v, K1v);
        K0 = K0v[0];
        K1 = K1v[0];
      } else if (ws > 0) {
        horner_y2_fibre<1>(base, in_estride, rowoff, f, L, yp, K0, K1);
      } else if (ws < 0) {
        horner_y2_fibre<-1>(base, in_estride, rowoff, f, L, yp, K0, K1);
      } else {
        horner_y2_fibre<0>(base, in_estride, rowoff, f, L, yp, K0, K1);
      }
      const int ro = __ldg(outpos + f);
      const int64_t o = (int64_t)ro * out_estride;
      if (live) out[i0 * out_nstride + o] = out_entry<A32C>(K0, bfL, ro);
      if (two) out[i1 * out_nstride + o] = out_entry<A32C>(K1, bfL, ro);
    }
  } else {
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const A32C::X &x = c == 0 ? x0 : x1;
      const float4 *base = in + (c == 0 ? p0 : p1) * in_nstride;
      const bool wr = c == 0 ? live : two;
      const int64_t node = c == 0 ? i0 : i1;
      for (int f = grp; f < st.nfib; f += G) {
        const int L = __ldg(st.fiblen + f);
        const float4 J = FM ? horner1_any<A32C>(base + __ldg(st.fiboff + f), 1, L, x)
                            : horner_any<A32C>(base, in_estride, rowoff, f, L, x);
        const int ro = __ldg(outpos + f);
        if (wr) out[node * out_nstride + (int64_t)ro * out_estride] = out_entry<A32C>(J, bfL, ro);
      }
    }
  }
}

// Stage d < k-1 in the certified binary32 arithmetic, two consecutive nodes per thread: warp w
// takes node pairs of chunk w % nchunk (64 nodes) and fibres g, g+G, ... (g = w / nchunk), as
// k_stage does with one node per lane.
template <bool FM>
__global__ void __launch_bounds__(kThreads, 6)
    k_stage_c(const StageDev st, const int32_t *__restrict__ lab, const int32_t *__restrict__ par,
              const float4 *__restrict__ in, int64_t in_estride, int64_t in_nstride,
              float4 *__restrict__ out, int64_t out_estride, int64_t out_nstride, int64_t nnodes,
              int64_t nchunk, int G, AxisGrid g, int bfL) {
  extern __shared__ int32_t s_rowoff[];
  for (int i = threadIdx.x; i <= st.maxlen; i += blockDim.x) s_rowoff[i] = st.rowoff[i];
  __syncthreads();
  const int64_t nwarps = nchunk * G;
  // the loop bound is the same for the 32 lanes of a warp, so the vote inside sees all of them
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); w < nwarps;
       w += (int64_t)gridDim.x * kWarpsPerBlock)
    stage_chunk_c<FM>(st, st.outpos, s_rowoff, lab, par, 0, in, in_estride, in_nstride, out, out_estride,
                  out_nstride, nnodes, w % nchunk, (int)(w / nchunk), G, g, bfL);
}

// k_stage_tma in the certified binary32 arithmetic, two children per thread: the children of
// one parent always share it, so every warp whose boxes do not straddle 0 runs sign-free.  The
// error bound advances step by step from the magnitudes of the partial values (A32C::step's
// recursion).  The summed bound of the leaves (bform_entry), applied to the stages' much longer
// chains, widens the curve's last-level band by 44-48% and does not pay: measured with the
// band going to the float-pair tier, the depth-1 stage took 4.77 instead of 4.59 ms per step
// (each staged group rewritten first) and the tier 1.86 instead of 1.55 ms.  With stage 0
// writing its blocks in that form (each entry's row and fibre length known per output fibre,
// no rewriting pass) the stage still took 4.89 instead of 4.72 ms, the band grew from 22 168
// to 32 678 boxes and the tier from 1.49 to 1.77 ms: the stage is not bound by its bound's
// arithmetic.
__global__ void __launch_bounds__(512)
    k_stage_tma_c(const StageDev st, const int32_t *__restrict__ lab,
                  const int32_t *__restrict__ pptr, const float4 *__restrict__ in,
                  float4 *__restrict__ out, int64_t out_estride, int64_t out_nstride, int G,
                  AxisGrid g, int bfL) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  float4 *s_blk = reinterpret_cast<float4 *>(smem + 128);
  const int64_t p = blockIdx.x / G;
  const StageGroup r = stage_group<16>(st, (int)(blockIdx.x % G), G);
  if (r.fb >= r.fe) return;  // an empty group (the same for the whole CTA)
  const int64_t c0 = __ldg(pptr + p), c1 = __ldg(pptr + p + 1);
  if (threadIdx.x == 0) stage_group_copy(in, p, st.blk_in, r, bar, s_blk);
  __syncthreads();
  if (!mbar_wait_bounded(bar, 0)) return;
  for (int64_t n0 = c0; n0 < c1; n0 += 2 * (int64_t)blockDim.x) {
    const int64_t na = n0 + 2 * threadIdx.x;
    const bool live = na < c1, two = na + 1 < c1;
    const int64_t i0 = live ? na : c1 - 1, i1 = two ? na + 1 : i0;
    const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
    const bool fast = x0.cls != 0 && x1.cls != 0;
    if (__all_sync(0xffffffffu, fast)) {
      const YPair yp = ypair(yleaf(x0), yleaf(x1));
      const int ws = warp_sign(yp);
      // each fibre's length, offset and output position loaded one fibre ahead
      int Ln = __ldg(st.fiblen + r.fb), fon = __ldg(st.fiboff + r.fb), ron = __ldg(st.outpos + r.fb);
      for (int f = r.fb; f < r.fe; ++f) {
        const int L = Ln, fo = fon, ro = ron;
        if (f + 1 < r.fe) {
          Ln = __ldg(st.fiblen + f + 1);
          fon = __ldg(st.fiboff + f + 1);
          ron = __ldg(st.outpos + f + 1);
        }
        const float4 *const b[2] = {s_blk + (fo - r.c_lo), nullptr};
        float4 K0[2], K1[2];
        if (ws > 0)
          horner_y2<1, 1>(b, L, yp, K0, K1);
        else if (ws < 0)
          horner_y2<1, -1>(b, L, yp, K0, K1);
        else
          horner_y2<1, 0>(b, L, yp, K0, K1);
        const int64_t o = (int64_t)ro * out_estride;
        if (live) out[i0 * out_nstride + o] = out_entry<A32C>(K0[0], bfL, ro);
        if (two) out[i1 * out_nstride + o] = out_entry<A32C>(K1[0], bfL, ro);
      }
    } else {
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        const A32C::X &x = c == 0 ? x0 : x1;
        const bool wr = c == 0 ? live : two;
        const int64_t node = c == 0 ? i0 : i1;
        for (int f = r.fb; f < r.fe; ++f) {
          const int L = __ldg(st.fiblen + f);
          const float4 J = horner1_any<A32C>(s_blk + (__ldg(st.fiboff + f) - r.c_lo), 1, L, x);
          const int ro = __ldg(st.outpos + f);
          if (wr) out[node * out_nstride + (int64_t)ro * out_estride] = out_entry<A32C>(J, bfL, ro);
        }
      }
    }
  }
}

// Where the leaf stage reads polynomial f's block for parent p: the parent blocks in global
// memory (node-major), or (StagedBlocks) consecutive parents' blocks staged in shared memory
// (separate types, so that each call site's loads are shared-memory or global ones).
struct GlobalBlocks {
  const LeafArgs &A;
  __device__ const float4 *operator()(int f, int64_t p) const {
    return (const float4 *)A.in[f] + p * A.blk[f];
  }
};

// The last stage of polynomials fb .. fe-1 on the leaf pair (i0, i1) with parents p0, p1
// (blocks from src), in the certified binary32 arithmetic, each decision ORed into the
// pair's state: ex[c] (some polynomial excludes leaf c) and am[c] (some decision is left to
// binary64).  A warp whose pairs each share a parent and do not straddle 0 takes the paired,
// sign-free path (two polynomials of one length at a time when NPMAX is 2); any other warp
// runs every leaf on its own.
template <int NPMAX, class Src, bool BF = false>
__device__ __forceinline__ void leaf_pair_eval(const LeafArgs &A, int fb, int fe, const Src &src,
                                               int64_t i0, int64_t i1, bool live, bool two,
                                               const A32C::X &x0, const A32C::X &x1, int64_t p0,
                                               int64_t p1, int64_t nleaves,
                                               double *__restrict__ lo, double *__restrict__ hi,
                                               bool (&ex)[2], bool (&am)[2]) {
  using V = float4;
  auto decide = [&](int f, int c, const V &J) {
    if (lo && live && (c == 0 || two)) {
      const int64_t i = c == 0 ? i0 : i1;
      lo[(int64_t)f * nleaves + i] = A32C::lo(J);
      hi[(int64_t)f * nleaves + i] = A32C::hi(J);
    }
    const int r = A32C::classify(J, A.rel[f]);
    ex[c] = ex[c] || r == 0;
    am[c] = am[c] || r == 2;
  };
  const bool fast = p0 == p1 && x0.cls != 0 && x1.cls != 0;
  if (__all_sync(0xffffffffu, fast)) {
    const YPair yp = ypair(yleaf(x0), yleaf(x1));
    const int ws = warp_sign(yp);
    int f = fb;
    if (NPMAX == 2) {
      for (; f + 1 < fe && A.len[f] == A.len[f + 1]; f += 2) {
        const V *const b[2] = {src(f, p0), src(f + 1, p0)};
        V K0[2], K1[2];
        if (ws > 0)
          horner_y2<2, 1, BF>(b, A.len[f], yp, K0, K1);
        else if (ws < 0)
          horner_y2<2, -1, BF>(b, A.len[f], yp, K0, K1);
        else
          horner_y2<2, 0, BF>(b, A.len[f], yp, K0, K1);
        decide(f, 0, K0[0]);
        decide(f + 1, 0, K0[1]);
        decide(f, 1, K1[0]);
        decide(f + 1, 1, K1[1]);
      }
    }
    for (; f < fe; ++f) {
      const V *const b[2] = {src(f, p0), nullptr};
      V K0[2], K1[2];
      if (ws > 0)
        horner_y2<1, 1, BF>(b, A.len[f], yp, K0, K1);
      else if (ws < 0)
        horner_y2<1, -1, BF>(b, A.len[f], yp, K0, K1);
      else
        horner_y2<1, 0, BF>(b, A.len[f], yp, K0, K1);
      decide(f, 0, K0[0]);
      decide(f, 1, K1[0]);
    }
  } else {
    // the leaf index c is a run-time value here: decisions go to a pair of registers, not to
    // ex[c] / am[c] (a dynamically indexed array would live in local memory)
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      const A32C::X &x = c == 0 ? x0 : x1;
      const int64_t p = c == 0 ? p0 : p1;
      bool e1 = false, a1 = false;
      auto decide1 = [&](int f, const V &J) {
        if (lo && live && (c == 0 || two)) {
          const int64_t i = c == 0 ? i0 : i1;
          lo[(int64_t)f * nleaves + i] = A32C::lo(J);
          hi[(int64_t)f * nleaves + i] = A32C::hi(J);
        }
        const int r = A32C::classify(J, A.rel[f]);
        e1 = e1 || r == 0;
        a1 = a1 || r == 2;
      };
      int f = fb;
      if (NPMAX == 2) {
        for (; f + 1 < fe && A.len[f] == A.len[f + 1]; f += 2) {
          V J0, J1;
          horner1x2_any<A32C>(src(f, p), src(f + 1, p), A.len[f], x, J0, J1);
          decide1(f, J0);
          decide1(f + 1, J1);
        }
      }
      for (; f < fe; ++f) decide1(f, horner1_any<A32C>(src(f, p), 1, A.len[f], x));
      if (c == 0) {
        ex[0] = ex[0] || e1;
        am[0] = am[0] || a1;
      } else {
        ex[1] = ex[1] || e1;
        am[1] = am[1] || a1;
      }
    }
  }
}

// keep (0 where some polynomial excludes the leaf) and flag (1 where the leaf is kept and some
// decision is left to binary64) of the leaf pair.
__device__ __forceinline__ void leaf_pair_store(int64_t i0, int64_t i1, bool live, bool two,
                                                const bool (&ex)[2], const bool (&am)[2],
                                                uint8_t *__restrict__ keep,
                                                uint8_t *__restrict__ flag) {
  if (live) {
    keep[i0] = ex[0] ? 0 : 1;
    if (flag) flag[i0] = (!ex[0] && am[0]) ? 1 : 0;
    if (two) {
      keep[i1] = ex[1] ? 0 : 1;
      if (flag) flag[i1] = (!ex[1] && am[1]) ? 1 : 0;
    }
  }
}

// The last stage and C0 of the leaf pair (i0, i1): every polynomial, then the decisions.
template <class Src>
__device__ __forceinline__ void leaf_pair_c(const LeafArgs &A, int npoly, const Src &src,
                                            int64_t i0, int64_t i1, bool live, bool two,
                                            const A32C::X &x0, const A32C::X &x1, int64_t p0,
                                            int64_t p1, int64_t nleaves,
                                            uint8_t *__restrict__ keep, double *__restrict__ lo,
                                            double *__restrict__ hi, uint8_t *__restrict__ flag,
                                            bool bf) {
  bool ex[2] = {false, false}, am[2] = {false, false};
  // bf: the parents' blocks carry the summed bound (a stage wrote them); the coefficient
  // block of a one-variable system does not
  if (bf)
    leaf_pair_eval<2, Src, true>(A, 0, npoly, src, i0, i1, live, two, x0, x1, p0, p1, nleaves,
                                 lo, hi, ex, am);
  else
    leaf_pair_eval<2, Src, false>(A, 0, npoly, src, i0, i1, live, two, x0, x1, p0, p1, nleaves,
                                  lo, hi, ex, am);
  leaf_pair_store(i0, i1, live, two, ex, am, keep, flag);
}

// One warp's share of k_leaf_c: the 32 leaf pairs of tile t (64 leaves).  par/poff as in
// leaf_item.
__device__ __forceinline__ void leaf_tile_c(const LeafArgs &A, int npoly,
                                            const int32_t *__restrict__ lab,
                                            const int32_t *__restrict__ par, int64_t poff,
                                            int64_t nleaves, int64_t t, const AxisGrid &g,
                                            uint8_t *__restrict__ keep, double *__restrict__ lo,
                                            double *__restrict__ hi, uint8_t *__restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t npairs = (nleaves + 1) >> 1;
  const int64_t q = t * 32 + lane;
  const bool live = q < npairs;  // a lane past the end repeats the last pair, stores nothing
  const int64_t i0 = 2 * (live ? q : npairs - 1);
  const bool two = i0 + 1 < nleaves;
  const int64_t i1 = two ? i0 + 1 : i0;
  const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
  const int64_t p0 = par ? (int64_t)__ldg(par + i0) - poff : 0;
  const int64_t p1 = par ? (int64_t)__ldg(par + i1) - poff : 0;
  leaf_pair_c(A, npoly, GlobalBlocks{A}, i0, i1, live, two, x0, x1, p0, p1, nleaves, keep, lo,
              hi, flag, par != nullptr);
}

__global__ void __launch_bounds__(kThreads, 6)
    k_leaf_c(LeafArgs A, int npoly, const int32_t *__restrict__ lab,
             const int32_t *__restrict__ par, int64_t nleaves, AxisGrid g,
             uint8_t *__restrict__ keep, double *__restrict__ lo, double *__restrict__ hi,
             uint8_t *__restrict__ flag) {
  const int64_t ntiles = (((nleaves + 1) >> 1) + 31) >> 5;
  // the loop bound is the same for the 32 lanes of a warp, so the vote inside sees all of them
  for (int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); t < ntiles;
       t += (int64_t)gridDim.x * kWarpsPerBlock)
    leaf_tile_c(A, npoly, lab, par, 0, nleaves, t, g, keep, lo, hi, flag);
}

// Leaf chunks of k_leaf_tma_c: kLeafIter pairs per thread, at most kLeafParents parents staged.
constexpr int kLeafIter = 2;
constexpr int kLeafParents = 8;

struct StagedBlocks {  // the staged blocks of parents p0 .. p0 + n - 1 (shared memory)
  const LeafArgs &A;
  const float4 *s_blk;
  const int32_t *s_off;
  int64_t p0;
  __device__ const float4 *operator()(int f, int64_t p) const {
    return s_blk + s_off[f] + (p - p0) * A.blk[f];
  }
};

// One thread: the bulk copies of parents pf .. pl's blocks, every polynomial's at s_off[f]
// (kLeafParents blocks apart), completing on bar.
__device__ __forceinline__ void leaf_chunk_copy(const LeafArgs &A, int npoly, int64_t pf,
                                                int64_t pl, uint64_t *bar, int32_t *s_off,
                                                float4 *s_blk) {
  mbar_init(bar, 1);
  const int64_t np = pl - pf + 1;
  int32_t o = 0;
  uint32_t total = 0;
  for (int f = 0; f < npoly; ++f) {
    s_off[f] = o;
    o += (int32_t)(kLeafParents * A.blk[f]);
    total += (uint32_t)(np * A.blk[f] * (int64_t)sizeof(float4));
  }
  mbar_arrive_expect_tx(bar, total);
  for (int f = 0; f < npoly; ++f) {
    const char *src = reinterpret_cast<const char *>((const float4 *)A.in[f] + pf * A.blk[f]);
    char *dst = reinterpret_cast<char *>(s_blk + s_off[f]);
    const uint64_t bytes = (uint64_t)(np * A.blk[f]) * sizeof(float4);
    for (uint64_t b = 0; b < bytes; b += 32768) {
      const uint32_t n = (uint32_t)(bytes - b < 32768 ? bytes - b : 32768);
      bulk_copy_g2s(dst + b, src + b, n, bar);
    }
  }
}

// k_leaf_c with the parents' blocks brought into shared memory by bulk copies (mbarrier,
// bounded wait): the CTA takes the leaves first .. last (at most 2 kLeafIter blockDim.x), two
// per thread per pass; their parents are consecutive nodes, whose node-major blocks are one
// contiguous range per polynomial, copied once when at most kLeafParents of them (else the
// CTA reads global memory as k_leaf_c does).  Parent indices minus poff index A's blocks.
__device__ __forceinline__ void leaf_tma_c_chunk(const LeafArgs &A, int npoly,
                                                 const int32_t *__restrict__ lab,
                                                 const int32_t *__restrict__ par, int64_t poff,
                                                 int64_t first, int64_t last, int64_t nleaves,
                                                 const AxisGrid &g, uint8_t *__restrict__ keep,
                                                 double *__restrict__ lo, double *__restrict__ hi,
                                                 uint8_t *__restrict__ flag, unsigned char *smem) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int32_t *s_off = reinterpret_cast<int32_t *>(smem + 16);
  float4 *s_blk = reinterpret_cast<float4 *>(smem + 128);
  const int64_t pf = __ldg(par + first) - poff, pl = __ldg(par + last) - poff;
  const bool staged = pl - pf < kLeafParents;
  if (staged) {
    if (threadIdx.x == 0) leaf_chunk_copy(A, npoly, pf, pl, bar, s_off, s_blk);
    __syncthreads();
    const bool ok = mbar_wait_bounded(bar, 0);
    if (!__syncthreads_and(ok)) return;
  }
  const StagedBlocks sb{A, s_blk, s_off, pf};
  const GlobalBlocks gb{A};
  // every warp runs the same trip count (the vote inside sees all 32 lanes); the blocks were
  // written for the summed bound (out_entry), staged or not
  for (int it = 0; it < kLeafIter; ++it) {
    const int64_t na = first + (int64_t)it * 2 * blockDim.x + 2 * threadIdx.x;
    const bool live = na <= last, two = na + 1 <= last;
    const int64_t i0 = live ? na : last, i1 = two ? na + 1 : i0;
    const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
    const int64_t p0 = __ldg(par + i0) - poff, p1 = __ldg(par + i1) - poff;
    bool ex[2] = {false, false}, am[2] = {false, false};
    if (staged)
      leaf_pair_eval<2, StagedBlocks, true>(A, 0, npoly, sb, i0, i1, live, two, x0, x1, p0, p1,
                                            nleaves, lo, hi, ex, am);
    else
      leaf_pair_eval<2, GlobalBlocks, true>(A, 0, npoly, gb, i0, i1, live, two, x0, x1, p0, p1,
                                            nleaves, lo, hi, ex, am);
    leaf_pair_store(i0, i1, live, two, ex, am, keep, flag);
  }
}

__global__ void __launch_bounds__(kThreads, 6)
    k_leaf_tma_c(LeafArgs A, int npoly, const int32_t *__restrict__ lab,
                 const int32_t *__restrict__ par, int64_t nleaves, AxisGrid g,
                 uint8_t *__restrict__ keep, double *__restrict__ lo, double *__restrict__ hi,
                 uint8_t *__restrict__ flag) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int64_t chunk = 2 * (int64_t)kLeafIter * blockDim.x;
  const int64_t first = (int64_t)blockIdx.x * chunk;
  const int64_t last = (first + chunk < nleaves ? first + chunk : nleaves) - 1;
  leaf_tma_c_chunk(A, npoly, lab, par, 0, first, last, nleaves, g, keep, lo, hi, flag, smem);
}

// k_leaf_tma_c for two or more polynomials, without the work that C0 makes useless: each
// thread runs polynomial 0 on its ITER pairs and settles the pairs whose leaves it excludes;
// the other pairs are queued in shared memory (warp-aggregated slots, so that the pairs of a
// warp stay neighbours) with their decisions so far, and the CTA's warps run the remaining
// polynomials on the queue.  C0 keeps a leaf only if no polynomial excludes it, so the
// decisions are those of k_leaf_tma_c; the leaves' interval values are not written.  The CTA
// takes the leaves first .. last (at most 2 ITER kThreads, ITER pairs per thread in the first
// phase); parent indices minus poff index A's blocks.
template <int ITER>
struct LeafQueue {
  int nq;
  int16_t q[ITER * kThreads];  // queued pair: its index in the chunk
  uint8_t st[ITER * kThreads]; // its decisions so far (ex0, am0, ex1, am1)
};

template <int ITER>
__device__ __forceinline__ void leaf_q_chunk(const LeafArgs &A, int npoly,
                                             const int32_t *__restrict__ lab,
                                             const int32_t *__restrict__ par, int64_t poff,
                                             int64_t first, int64_t last, const AxisGrid &g,
                                             uint8_t *__restrict__ keep,
                                             uint8_t *__restrict__ flag, unsigned char *smem,
                                             LeafQueue<ITER> &Q) {
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  int32_t *s_off = reinterpret_cast<int32_t *>(smem + 16);
  float4 *s_blk = reinterpret_cast<float4 *>(smem + 128);
  const int64_t pf = __ldg(par + first) - poff, pl = __ldg(par + last) - poff;
  const bool staged = pl - pf < kLeafParents;
  if (threadIdx.x == 0) {
    Q.nq = 0;
    if (staged) leaf_chunk_copy(A, npoly, pf, pl, bar, s_off, s_blk);
  }
  __syncthreads();
  const bool ok = !staged || mbar_wait_bounded(bar, 0);
  if (!__syncthreads_and(ok)) return;
  // the blocks were written for the summed bound (out_entry), staged or not
  const StagedBlocks sb{A, s_blk, s_off, pf};
  const GlobalBlocks gb{A};
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < ITER; ++it) {
    const int q = it * kThreads + (int)threadIdx.x;
    const int64_t na = first + 2 * (int64_t)q;
    const bool live = na <= last, two = na + 1 <= last;
    const int64_t i0 = live ? na : last, i1 = two ? na + 1 : i0;
    const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
    const int64_t p0 = __ldg(par + i0) - poff, p1 = __ldg(par + i1) - poff;
    bool ex[2] = {false, false}, am[2] = {false, false};
    if (staged)
      leaf_pair_eval<1, StagedBlocks, true>(A, 0, 1, sb, i0, i1, live, two, x0, x1, p0, p1, 0,
                                            nullptr, nullptr, ex, am);
    else
      leaf_pair_eval<1, GlobalBlocks, true>(A, 0, 1, gb, i0, i1, live, two, x0, x1, p0, p1, 0,
                                            nullptr, nullptr, ex, am);
    const bool more = live && !(ex[0] && (ex[1] || !two));
    if (live && !more) leaf_pair_store(i0, i1, live, two, ex, am, keep, flag);
    const unsigned m = __ballot_sync(0xffffffffu, more);
    int base = 0;
    if (lane == 0 && m != 0u) base = atomicAdd(&Q.nq, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (more) {
      const int slot = base + __popc(m & ((1u << lane) - 1u));
      Q.q[slot] = (int16_t)q;
      Q.st[slot] = (uint8_t)((ex[0] ? 1 : 0) | (am[0] ? 2 : 0) | (ex[1] ? 4 : 0) | (am[1] ? 8 : 0));
    }
  }
  __syncthreads();
  const int nq = Q.nq;
  // the loop bound is the same for the 32 lanes of a warp (the votes inside see all of them);
  // a lane past the queue's end repeats its last pair and stores nothing
  for (int b = (int)(threadIdx.x & ~31u); b < nq; b += kThreads) {
    const bool in = b + lane < nq;
    const int sl = in ? b + lane : nq - 1;
    const int q = Q.q[sl], st = Q.st[sl];
    const int64_t i0 = first + 2 * (int64_t)q;
    const bool two = i0 + 1 <= last;
    const int64_t i1 = two ? i0 + 1 : i0;
    const A32C::X x0 = A32C::box(g, __ldg(lab + i0)), x1 = A32C::box(g, __ldg(lab + i1));
    const int64_t p0 = __ldg(par + i0) - poff, p1 = __ldg(par + i1) - poff;
    bool ex[2] = {(st & 1) != 0, (st & 4) != 0}, am[2] = {(st & 2) != 0, (st & 8) != 0};
    if (staged)
      leaf_pair_eval<1, StagedBlocks, true>(A, 1, npoly, sb, i0, i1, in, two, x0, x1, p0, p1, 0,
                                            nullptr, nullptr, ex, am);
    else
      leaf_pair_eval<1, GlobalBlocks, true>(A, 1, npoly, gb, i0, i1, in, two, x0, x1, p0, p1, 0,
                                            nullptr, nullptr, ex, am);
    leaf_pair_store(i0, i1, in, two, ex, am, keep, flag);
  }
}

template <int ITER>
__global__ void __launch_bounds__(kThreads, 8)
    k_leaf_tma_q(LeafArgs A, int npoly, const int32_t *__restrict__ lab,
                 const int32_t *__restrict__ par, int64_t nleaves, AxisGrid g,
                 uint8_t *__restrict__ keep, uint8_t *__restrict__ flag) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ LeafQueue<ITER> Q;
  const int64_t chunk = 2 * (int64_t)ITER * kThreads;
  const int64_t first = (int64_t)blockIdx.x * chunk;
  const int64_t last = (first + chunk < nleaves ? first + chunk : nleaves) - 1;
  leaf_q_chunk<ITER>(A, npoly, lab, par, 0, first, last, g, keep, flag, smem, Q);
}

int leaf_tma_grid(int64_t leaves, int iter = kLeafIter) {
  const int64_t chunk = 2 * (int64_t)iter * kThreads;
  return (int)((leaves + chunk - 1) / chunk);
}

int leaf_pair_grid(int64_t leaves) {
  int64_t b = ((leaves + 1) / 2 + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count() * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

constexpr size_t kMaxDynSmem = 200 * 1024;
// a staged stage's CTA holds at most about this much of its parent's block (fibre groups)
constexpr int64_t kStageGroupBytes = 48 * 1024;
// depths with at least this many nodes, or this many multiply-adds per node, run the
// certified stage two nodes per thread
constexpr int64_t kPairNodes = 65536;

// The input of stage d >= 1 (the output of stage d-1) is node-major iff stage d is the leaf
// stage or is TMA-staged; a non-staged inner stage reads it entry-major.
inline bool tma_input_node_major(int d, int k, const bool *tma) { return d + 1 == k || tma[d]; }

int leaf_grid(int64_t items) {
  int64_t b = (items + kThreads - 1) / kThreads;
  const int64_t cap = (int64_t)sm_count() * 32;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// Bytes of one depth's partial-evaluation block (n nodes of blk entries), rounded up to 256 so
// that the next block starts on a 256-byte boundary.
template <class AR>
size_t block_bytes(int64_t n, int64_t blk) {
  return ((size_t)n * (size_t)blk * sizeof(typename AR::V) + 255) & ~(size_t)255;
}

// Bytes of partial-evaluation blocks a level needs (each block 256-byte aligned).
template <class AR>
size_t level_scratch_bytes(const SysDev &sys, const CsfView &c) {
  size_t total = 0;
  for (int f = 0; f < sys.npoly; ++f)
    for (int d = 0; d + 1 < sys.k; ++d) total += block_bytes<AR>(c.N[d], sys.p[f].st[d].blk_out);
  return total;
}

// ---------------------------------------------------------------------------------------
// Autotuner: a stage or leaf launch has a few variants that compute the same outputs (one or
// two nodes per thread, fibre-group counts, CTA sizes).  The first launch of a shape key
// (arithmetic, depth, log2 of the node counts, fibre length, log2 of the fibre count) times
// every variant on the real data, CUDA events on the launching stream, and keeps the fastest;
// later launches of that key use it.  The last variant timed leaves the outputs in place.
// ---------------------------------------------------------------------------------------
struct Tuner {
  std::mutex mu;
  std::unordered_map<uint64_t, int> best;
  int mode = 1;      // 0: heuristic variant 0 only, 1: tune, 2 + v: variant v wherever it exists
  std::string path;  // cache file ("" = in memory only)
};
Tuner &tuner() {
  static Tuner t;
  return t;
}

int ilog2(int64_t x) {
  int r = 0;
  while (x > 1) {
    x >>= 1;
    ++r;
  }
  return r;
}

uint64_t tune_key(int kind, int arith, int d, int64_t n, int64_t nparent, int maxlen, int nfib) {
  return ((uint64_t)(kind & 0xF) << 60) | ((uint64_t)(arith & 0xF) << 56) |
         ((uint64_t)(d & 0xF) << 52) | ((uint64_t)(ilog2(n + 1) & 0x3F) << 46) |
         ((uint64_t)(ilog2(nparent + 1) & 0x3F) << 40) | ((uint64_t)(maxlen & 0xFFFF) << 24) |
         ((uint64_t)(ilog2(nfib + 1) & 0x3F) << 18);
}

// Runs launch(v) for the cached variant of `key`, or times variants 0..nvar-1 and caches the
// fastest.  launch returns a status; the stream is synchronised only while tuning.
template <class F>
int tuned_launch(uint64_t key, int nvar, cudaStream_t s, F launch) {
  Tuner &T = tuner();
  int v = -1;
  {
    std::lock_guard<std::mutex> g(T.mu);
    if (T.mode == 0 || nvar <= 1) v = 0;
    else if (T.mode >= 2) v = T.mode - 2 < nvar ? T.mode - 2 : 0;
    else {
      auto it = T.best.find(key);
      if (it != T.best.end()) v = it->second < nvar ? it->second : 0;
    }
  }
  if (v >= 0) return launch(v);
  cudaEvent_t a = nullptr, b = nullptr;
  VX_CUDA(cudaEventCreate(&a));
  VX_CUDA(cudaEventCreate(&b));
  float bestms = 0.f;
  int bestv = 0, rc = VX_OK;
  for (int c = 0; c < nvar && rc == VX_OK; ++c) {
    cudaEventRecord(a, s);
    rc = launch(c);
    cudaEventRecord(b, s);
    float ms = 0.f;
    if (rc == VX_OK && (cudaEventSynchronize(b) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, a, b) != cudaSuccess)) {
      set_error("autotune timing failed");
      rc = VX_ECUDA;
    }
    if (rc == VX_OK && (c == 0 || ms < bestms)) {
      bestms = ms;
      bestv = c;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != VX_OK) return rc;
  // the outputs of the last variant are in place; run the best one if it was not the last so
  // that every output comes from one variant
  if (bestv != nvar - 1) rc = launch(bestv);
  std::lock_guard<std::mutex> g(T.mu);
  T.best[key] = bestv;
  if (!T.path.empty()) {
    if (FILE *fp = std::fopen(T.path.c_str(), "a")) {
      std::fprintf(fp, "%llx %d\n", (unsigned long long)key, bestv);
      std::fclose(fp);
    }
  }
  return rc;
}

// ext_scratch != nullptr: the blocks are carved from it (ext_bytes long) and nothing is allocated.
template <class AR>
// pgrid (nullable): polynomial f's stages use pgrid[f] (point or box grids for the Taylor
// form); tl (nullable, binary64 only): the leaves combine the polynomials into the Taylor form
// instead of testing each one.
int eval_level_t(const SysDev &sys, const CsfView &c, const LevelGrid &grid, double *d_lo,
                 double *d_hi, uint8_t *d_keep, uint8_t *d_flag, float theta, cudaStream_t s,
                 Timer *tm, int64_t *madds_out, int kind0, void *ext_scratch = nullptr,
                 size_t ext_bytes = 0, const LevelGrid *pgrid = nullptr,
                 const TaylorLeaf *tl = nullptr) {
  using V = typename AR::V;
  const int k = sys.k;
  const int64_t nleaves = c.N[k - 1];
  int64_t madds = 0;
  if (nleaves == 0) {
    if (madds_out) *madds_out = 0;
    return VX_OK;
  }
  // blocks of depths 0..k-2, one allocation per polynomial
  void *mem[VX_MAXPOLY] = {nullptr};
  V *buf[VX_MAXPOLY][VX_KMAX] = {{nullptr}};
  int rc = VX_OK;
  if (ext_scratch) {
    if (level_scratch_bytes<AR>(sys, c) > ext_bytes) {
      set_error("the level needs %zu bytes of scratch, more than the %zu available",
                level_scratch_bytes<AR>(sys, c), ext_bytes);
      return VX_ECAPACITY;
    }
    char *p = (char *)ext_scratch;
    for (int f = 0; f < sys.npoly; ++f)
      for (int d = 0; d + 1 < k; ++d) {
        buf[f][d] = (V *)p;
        p += block_bytes<AR>(c.N[d], sys.p[f].st[d].blk_out);
      }
  }
  // one allocation per polynomial, each depth's block starting on a 256-byte boundary (the
  // bulk copies of the staged kernels read parent blocks from 16-byte aligned addresses)
  for (int f = 0; f < sys.npoly && rc == VX_OK && !ext_scratch; ++f) {
    size_t total = 0;
    for (int d = 0; d + 1 < k; ++d) total += block_bytes<AR>(c.N[d], sys.p[f].st[d].blk_out);
    if (total == 0) continue;
    rc = dmalloc(&mem[f], total, s);
    char *p = (char *)mem[f];
    for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
      buf[f][d] = (V *)p;
      p += block_bytes<AR>(c.N[d], sys.p[f].st[d].blk_out);
    }
  }

  for (int f = 0; f < sys.npoly && rc == VX_OK; ++f) {
    const LevelGrid &pg = pgrid ? pgrid[f] : grid;
    // stage d (1 <= d < k-1) stages its parents' blocks by TMA when the depth has enough
    // nodes to fill the GPU with 128-node CTAs and two parent blocks fit in shared memory
    bool tma[VX_KMAX] = {false};
    for (int d = 1; d + 1 < k; ++d) {
      const StageDev &st = sys.p[f].st[d];
      // cp.async.bulk needs 16-byte aligned source and size: every parent block must start on
      // a 16-byte boundary (the buffer itself is 256-byte aligned), and a group's range widened
      // to 16-byte boundaries must stay inside its block
      const bool aligned = (st.blk_in * (int64_t)sizeof(V)) % 16 == 0 &&
                           (reinterpret_cast<uintptr_t>(buf[f][d - 1]) & 15u) == 0;
      if (aligned && c.N[d] >= 16384 && c.N[d] >= 128 * c.N[d - 1]) tma[d] = true;
    }
    for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
      // a stage whose consumer stages its parents' blocks writes them fibre-major
      StageDev st = sys.p[f].st[d];
      if (tma[d + 1]) st.outpos = st.outpos_fm;
      const int64_t w = c.N[d] * (st.blk_in - st.nfib);
      madds += w;
      // node-major output when the consumer is the leaf stage or a TMA-staged stage
      const bool node_major = d + 2 == k || tma[d + 1];
      // certified binary32 leaves (not the Taylor form's) read their parents' blocks already
      // rewritten for the summed bound
      const int bfL = std::is_same<AR, A32C>::value && !tl && d + 2 == k ? (int)st.blk_out : 0;
      const int64_t oe = node_major ? 1 : c.N[d], on = node_major ? st.blk_out : 1;
      if (tm && tm->on) rc = tm->begin(d == 0 ? kind0 : kind0 + 1, w);
      if (rc != VX_OK) break;
      const V *in = d == 0 ? AR::coef(sys.p[f]) : buf[f][d - 1];
      const int arith = std::is_same<AR, A64>::value ? 0 : (std::is_same<AR, A32>::value ? 1 : 2);
      if (tma[d]) {
        // the same value from every caller: host threads launching concurrently never lower
        // the limit below another one's need
        if (cudaFuncSetAttribute(k_stage_tma<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_stage_tma_c, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxDynSmem) != cudaSuccess) {
          set_error("cudaFuncSetAttribute(shared memory %zu) failed", kMaxDynSmem);
          rc = VX_ECUDA;
          break;
        }
        // one CTA per (parent, fibre group), threads ~ the average number of children; the
        // groups are at least enough for a CTA's share of the block to stay within
        // kStageGroupBytes (several CTAs per SM) and for the launch to fill the GPU.
        // Variants: 0 the heuristic (two children per thread in the certified binary32
        // arithmetic), 1 one child per thread, 2 twice the fibre groups, 3 half the threads
        const int64_t np = c.N[d - 1];
        const int64_t avg = c.N[d] / np;
        const int threads0 = avg >= 512 ? 512 : (avg >= 256 ? 256 : 128);
        const int64_t gsm = ((int64_t)(st.blk_in * sizeof(V)) + kStageGroupBytes - 1) / kStageGroupBytes;
        int64_t G0 = std::max<int64_t>(((int64_t)sm_count() * 8 + np - 1) / np, gsm);
        if (G0 > st.nfib) G0 = st.nfib;
        if (G0 < 1) G0 = 1;
        // a group holds fewer than blk_in / G + maxlen entries, plus one at each end for the
        // 16-byte widening
        auto smem_of = [&](int64_t G) {
          return (size_t)128 + (size_t)((st.blk_in + G - 1) / G + st.maxlen + 2) * sizeof(V);
        };
        auto launch = [&](int v) -> int {
          int threads = threads0;
          int64_t G = G0;
          if (v == 2) G = std::min<int64_t>(st.nfib, 2 * G0);
          if (v == 3) threads = std::max(128, threads0 / 2);
          const size_t sm = smem_of(G);
          if (sm > kMaxDynSmem) {
            set_error("a stage's fibre group needs %zu bytes of shared memory", sm);
            return VX_EINVAL;
          }
          const bool two = std::is_same<AR, A32C>::value && v != 1;
          if (two)
            k_stage_tma_c<<<(unsigned)(np * G), threads, sm, s>>>(
                st, c.lab[d], c.ptr[d - 1], (const float4 *)in, (float4 *)buf[f][d], oe, on,
                (int)G, pg.ax[d], bfL);
          else
            k_stage_tma<AR><<<(unsigned)(np * G), threads, sm, s>>>(
                st, c.lab[d], c.ptr[d - 1], in, buf[f][d], oe, on, (int)G, pg.ax[d], bfL);
          note_launch();
          VX_LAUNCH_CHECK();
          return VX_OK;
        };
        rc = tuned_launch(tune_key(1, arith, d, c.N[d], np, st.maxlen, st.nfib), 4, s, launch);
      } else {
        // fibre groups: enough warps to fill the GPU several times over (a warp takes 32
        // nodes; 64 in the certified binary32 arithmetic when the depth has enough nodes for
        // the shared loads to pay).  Variants: 0 the heuristic, 1 the other node count per
        // warp (certified binary32), 2 four times the fibre groups, 3 (certified binary32)
        // sixteen times (stages with few nodes, such as stage 0, wait on their fibres' loads:
        // more warps hide more of that latency)
        const bool pairs0 = std::is_same<AR, A32C>::value &&
                            (c.N[d] >= kPairNodes || st.blk_in - st.nfib >= kPairNodes);
        const int64_t in_estride = d == 0 ? 1 : (tma_input_node_major(d, k, tma) ? 1 : c.N[d - 1]);
        const int64_t in_nstride = d == 0 ? 0 : (tma_input_node_major(d, k, tma) ? st.blk_in : 1);
        auto launch = [&](int vv) -> int {
          const int v = std::is_same<AR, A32C>::value ? vv : (vv == 1 ? 2 : 0);
          const int64_t G_mult = v == 3 ? 16 : (v == 2 ? 4 : 1);
          const bool pairs = v == 1 ? !pairs0 : pairs0;
          const int64_t per_warp = pairs ? 64 : 32;
          const int64_t nchunk = (c.N[d] + per_warp - 1) / per_warp;
          const int64_t target = (int64_t)sm_count() * 64 * G_mult;
          int64_t G = (target + nchunk - 1) / nchunk;
          if (G > st.nfib) G = st.nfib;
          if (G < 1) G = 1;
          int64_t blocks = (nchunk * G + kWarpsPerBlock - 1) / kWarpsPerBlock;
          if (blocks > (int64_t)sm_count() * 64) blocks = (int64_t)sm_count() * 64;
          // stage 0: the fibre-major copy of the coefficient block (consecutive loads along
          // a fibre, where the row-major block has one cache line per step)
          const V *fm0 = d == 0 ? AR::coef_fm(sys.p[f]) : nullptr;
          if (pairs && fm0)
            k_stage_c<true><<<(unsigned)blocks, kThreads, (st.maxlen + 1) * sizeof(int32_t), s>>>(
                st, c.lab[d], nullptr, (const float4 *)fm0, 1, 0, (float4 *)buf[f][d], oe, on,
                c.N[d], nchunk, (int)G, pg.ax[d], bfL);
          else if (fm0)
            k_stage<AR, true><<<(unsigned)blocks, kThreads, (st.maxlen + 1) * sizeof(int32_t), s>>>(
                st, c.lab[d], nullptr, fm0, 1, 0, buf[f][d], oe, on, c.N[d], nchunk, (int)G,
                pg.ax[d], bfL);
          else if (pairs)
            k_stage_c<false><<<(unsigned)blocks, kThreads, (st.maxlen + 1) * sizeof(int32_t), s>>>(
                st, c.lab[d], d == 0 ? nullptr : c.par[d], (const float4 *)in, in_estride,
                in_nstride, (float4 *)buf[f][d], oe, on, c.N[d], nchunk, (int)G, pg.ax[d], bfL);
          else
            k_stage<AR><<<(unsigned)blocks, kThreads, (st.maxlen + 1) * sizeof(int32_t), s>>>(
                st, c.lab[d], d == 0 ? nullptr : c.par[d], in, in_estride, in_nstride,
                buf[f][d], oe, on, c.N[d], nchunk, (int)G, pg.ax[d], bfL);
          note_launch();
          VX_LAUNCH_CHECK();
          return VX_OK;
        };
        rc = tuned_launch(tune_key(2, arith, d, c.N[d], d > 0 ? c.N[d - 1] : 0, st.maxlen,
                                   st.nfib),
                          std::is_same<AR, A32C>::value ? 4 : 2, s, launch);
      }
      if (rc != VX_OK) break;
      if (tm && tm->on) rc = tm->end();
    }
  }
  if (rc == VX_OK) {
    LeafArgs A{};
    int64_t wl = 0;
    for (int f = 0; f < sys.npoly; ++f) {
      const StageDev &st = sys.p[f].st[k - 1];
      A.rel[f] = sys.rel[f];
      A.in[f] = k == 1 ? (const void *)AR::coef(sys.p[f]) : (const void *)buf[f][k - 2];
      A.blk[f] = k == 1 ? 0 : st.blk_in;
      A.len[f] = st.maxlen;
      wl += nleaves * (st.blk_in - 1);
    }
    madds += wl;
    if (tm && tm->on) rc = tm->begin(kind0 + 2, wl);
    if (rc == VX_OK) {
      // variants (certified binary32): 0 two leaves per thread, 1 one leaf per thread, 2 two
      // leaves per thread with the parents' blocks staged in shared memory (CTA = 512
      // consecutive leaves; when the blocks fit), 3 / 4 the same skipping what C0 makes
      // useless, with 512 / 1024 leaves per CTA (2048 measured no faster)
      size_t leaf_smem = 128;
      for (int f = 0; f < sys.npoly; ++f)
        leaf_smem += (size_t)kLeafParents * (size_t)A.blk[f] * sizeof(float4);
      const bool leaf_tma = std::is_same<AR, A32C>::value && k >= 2 && leaf_smem <= kMaxDynSmem;
      // 3: k_leaf_tma_q (two or more polynomials, decisions only)
      const bool leaf_q = leaf_tma && sys.npoly >= 2 && d_lo == nullptr;
      if (leaf_tma &&
          (cudaFuncSetAttribute(k_leaf_tma_c, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxDynSmem) != cudaSuccess ||
           cudaFuncSetAttribute(k_leaf_tma_q<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxDynSmem) != cudaSuccess ||
           cudaFuncSetAttribute(k_leaf_tma_q<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kMaxDynSmem) != cudaSuccess)) {
        set_error("cudaFuncSetAttribute(shared memory %zu) failed", leaf_smem);
        rc = VX_ECUDA;
      }
      auto launch = [&](int v) -> int {
        if (std::is_same<AR, A32C>::value && v == 3)
          k_leaf_tma_q<2><<<(unsigned)leaf_tma_grid(nleaves, 2), kThreads, leaf_smem, s>>>(
              A, sys.npoly, c.lab[k - 1], c.par[k - 1], nleaves, grid.ax[k - 1], d_keep, d_flag);
        else if (std::is_same<AR, A32C>::value && v == 4)
          k_leaf_tma_q<4><<<(unsigned)leaf_tma_grid(nleaves, 4), kThreads, leaf_smem, s>>>(
              A, sys.npoly, c.lab[k - 1], c.par[k - 1], nleaves, grid.ax[k - 1], d_keep, d_flag);
        else if (std::is_same<AR, A32C>::value && v == 2)
          k_leaf_tma_c<<<(unsigned)leaf_tma_grid(nleaves), kThreads, leaf_smem, s>>>(
              A, sys.npoly, c.lab[k - 1], c.par[k - 1], nleaves, grid.ax[k - 1], d_keep, d_lo,
              d_hi, d_flag);
        else if (std::is_same<AR, A32C>::value && v == 0)
          k_leaf_c<<<leaf_pair_grid(nleaves), kThreads, 0, s>>>(
              A, sys.npoly, c.lab[k - 1], k == 1 ? nullptr : c.par[k - 1], nleaves,
              grid.ax[k - 1], d_keep, d_lo, d_hi, d_flag);
        else
          k_leaf<AR><<<leaf_grid(nleaves), kThreads, 0, s>>>(A, sys.npoly, c.lab[k - 1],
                                                            k == 1 ? nullptr : c.par[k - 1],
                                                            nleaves, grid.ax[k - 1], d_keep,
                                                            d_lo, d_hi, d_flag, theta);
        note_launch();
        VX_LAUNCH_CHECK();
        return VX_OK;
      };
      const int arith = std::is_same<AR, A64>::value ? 0 : (std::is_same<AR, A32>::value ? 1 : 2);
      if (tl) {
        if constexpr (std::is_same<AR, A64>::value) {
          AxisGrid gp = grid.ax[k - 1];
          gp.point = 1;
          gp.fexact = 0;
          k_leaf_taylor<<<leaf_grid(nleaves), kThreads, 0, s>>>(
              A, c.lab[k - 1], k == 1 ? nullptr : c.par[k - 1], nleaves, grid.ax[k - 1], gp, *tl,
              d_keep);
          note_launch();
          if (cudaGetLastError() != cudaSuccess) {
            set_error("Taylor leaf launch failed");
            rc = VX_ECUDA;
          }
        } else if constexpr (std::is_same<AR, A32C>::value) {
          AxisGrid gp = grid.ax[k - 1];
          gp.point = 1;  // binary32-exact centres when the grid's half points are (fexact)
          k_leaf_taylor_c<<<leaf_grid(nleaves), kThreads, 0, s>>>(
              A, c.lab[k - 1], k == 1 ? nullptr : c.par[k - 1], nleaves, grid.ax[k - 1], gp, *tl,
              d_keep);
          note_launch();
          if (cudaGetLastError() != cudaSuccess) {
            set_error("Taylor leaf launch failed");
            rc = VX_ECUDA;
          }
        } else {
          set_error("the Taylor form is evaluated in binary64 or certified binary32 only");
          rc = VX_EINVAL;
        }
      } else {
        if (rc == VX_OK)
          rc = tuned_launch(tune_key(3, arith, k - 1, nleaves, k > 1 ? c.N[k - 2] : 0,
                                     sys.p[0].st[k - 1].maxlen, sys.npoly),
                            std::is_same<AR, A32C>::value ? (leaf_q ? 5 : leaf_tma ? 3 : 2) : 1,
                            s, launch);
      }
      if (rc == VX_OK && tm && tm->on) rc = tm->end();
    }
  }
  for (int f = 0; f < sys.npoly; ++f) dfree(mem[f], s);
  if (madds_out) *madds_out = madds;
  return rc;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// Forests: the trees of many independent systems at one level, stored one after another at
// every depth (tree s owns depth-d nodes off[d][s] .. off[d][s+1]-1; parents index the whole
// forest).  One launch per depth evaluates every tree's nodes with its own system, grid and
// blocks: thread = node, every polynomial and fibre in turn.
// ---------------------------------------------------------------------------------------
namespace {

__device__ __forceinline__ int tree_of(const int64_t *__restrict__ off, int S, int64_t i) {
  int lo = 0, hi = S;  // largest s with off[s] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Depth d < k-1 of a forest: a queue of warp tasks, tree t owning tasks tasks[t] ..
// tasks[t+1]-1 (nchunk_t node chunks x G fibre groups); each task runs k_stage's (or
// k_stage_c's) warp body on its tree's nodes with the tree's polynomials, grid and
// node-major blocks.
template <class AR, bool PAIRS>
__global__ void __launch_bounds__(kThreads, 6)
    k_fstage(const ForestTree *__restrict__ trees, const int64_t *__restrict__ off, int S, int d,
             CsfView c, void *const *__restrict__ blk, const int64_t *__restrict__ tasks, int G) {
  using V = typename AR::V;
  constexpr bool FMF = std::is_same<AR, A32C>::value;
  const int k = c.k;
  const int64_t *offd = off + (int64_t)d * (S + 1);
  const int64_t *offp = off + (int64_t)(d > 0 ? d - 1 : 0) * (S + 1);
  const int64_t ntask = __ldg(tasks + S);
  // the task index is the same for the 32 lanes of a warp
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); w < ntask;
       w += (int64_t)gridDim.x * kWarpsPerBlock) {
    const int t = tree_of(tasks, S, w);
    const ForestTree &T = trees[t];
    const int64_t o = __ldg(offd + t), n = __ldg(offd + t + 1) - o;
    const int64_t per = PAIRS ? 64 : 32, nchunk = (n + per - 1) / per;
    const int64_t wl = w - __ldg(tasks + t);
    const int64_t chunk = wl % nchunk;
    const int grp = (int)(wl / nchunk);
    const int32_t *lab = c.lab[d] + o;
    const int32_t *par = d > 0 ? c.par[d] + o : nullptr;
    const int64_t poff = d > 0 ? __ldg(offp + t) : 0;
    for (int f = 0; f < T.dev.npoly; ++f) {
      const StageDev &st = T.dev.p[f].st[d];
      // stage 0 reads the coefficient block's fibre-major copy; certified binary32 also
      // writes and reads the inner stages' blocks fibre-major
      const int32_t *outpos = FMF && d + 2 < k ? st.outpos_fm : st.outpos;
      const bool fmr = d == 0 || FMF;
      const int bfL = FMF && d + 2 == k ? (int)st.blk_out : 0;  // the leaves' summed bound
      const V *in = d == 0 ? AR::coef_fm(T.dev.p[f])
                           : (const V *)blk[((int64_t)t * VX_MAXPOLY + f) * VX_KMAX + d - 1];
      V *out = (V *)blk[((int64_t)t * VX_MAXPOLY + f) * VX_KMAX + d];
      const int64_t in_nstride = d == 0 ? 0 : st.blk_in;
      if constexpr (PAIRS) {
        if (fmr)
          stage_chunk_c<true>(st, outpos, st.rowoff, lab, par, poff, (const float4 *)in, 1, in_nstride,
                              (float4 *)out, 1, st.blk_out, n, chunk, grp, G, T.ax[d], bfL);
        else
          stage_chunk_c<false>(st, outpos, st.rowoff, lab, par, poff, (const float4 *)in, 1, in_nstride,
                               (float4 *)out, 1, st.blk_out, n, chunk, grp, G, T.ax[d], bfL);
      } else {
        if (fmr)
          stage_chunk<AR, true>(st, outpos, st.rowoff, lab, par, poff, in, 1, in_nstride, out, 1,
                                st.blk_out, n, chunk, grp, G, T.ax[d], bfL);
        else
          stage_chunk<AR, false>(st, outpos, st.rowoff, lab, par, poff, in, 1, in_nstride, out, 1,
                                 st.blk_out, n, chunk, grp, G, T.ax[d], bfL);
      }
    }
  }
}

// The leaves of a forest: tree t owns warp tasks tasks[t] .. tasks[t+1]-1, each 32 leaves
// (64 in pairs for the certified binary32 arithmetic, k_leaf_c's body), with the tree's
// polynomials, grid and parent blocks.
template <class AR, bool PAIRS>
__global__ void __launch_bounds__(kThreads)
    k_fleaf(const ForestTree *__restrict__ trees, const int64_t *__restrict__ off, int S,
            CsfView c, void *const *__restrict__ blk, const int64_t *__restrict__ tasks,
            uint8_t *__restrict__ keep, uint8_t *__restrict__ flag, float theta) {
  const int k = c.k;
  const int64_t *offl = off + (int64_t)(k - 1) * (S + 1);
  const int64_t *offp = off + (int64_t)(k > 1 ? k - 2 : 0) * (S + 1);
  const int64_t ntask = __ldg(tasks + S);
  for (int64_t w = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5); w < ntask;
       w += (int64_t)gridDim.x * kWarpsPerBlock) {
    const int t = tree_of(tasks, S, w);
    const ForestTree &T = trees[t];
    const int64_t o = __ldg(offl + t), n = __ldg(offl + t + 1) - o;
    LeafArgs A;
    const int npoly = T.dev.npoly;
    for (int f = 0; f < npoly; ++f) {
      const StageDev &st = T.dev.p[f].st[k - 1];
      A.rel[f] = T.dev.rel[f];
      A.in[f] = k == 1 ? (const void *)AR::coef(T.dev.p[f])
                       : blk[((int64_t)t * VX_MAXPOLY + f) * VX_KMAX + k - 2];
      A.blk[f] = k == 1 ? 0 : st.blk_in;
      A.len[f] = st.maxlen;
    }
    const int32_t *lab = c.lab[k - 1] + o;
    const int32_t *par = k > 1 ? c.par[k - 1] + o : nullptr;
    const int64_t poff = k > 1 ? __ldg(offp + t) : 0;
    const int64_t wl = w - __ldg(tasks + t);
    if constexpr (PAIRS) {
      leaf_tile_c(A, npoly, lab, par, poff, n, wl, T.ax[k - 1], keep + o, nullptr, nullptr,
                  flag ? flag + o : nullptr);
    } else {
      const int64_t i = wl * 32 + (threadIdx.x & 31);
      if (i < n)
        leaf_item<AR>(A, npoly, lab, par, poff, i, n, T.ax[k - 1], keep + o, nullptr, nullptr,
                      flag ? flag + o : nullptr, theta);
    }
  }
}

// The leaves of a forest in the certified binary32 arithmetic with the single-system leaf
// kernels' bodies: CTA b takes chunk b - ctasks[t] of tree t's leaves (tree t owning CTAs
// ctasks[t] .. ctasks[t+1]-1), stages the chunk's parent blocks of the tree's own polynomials
// in shared memory and runs k_leaf_tma_q's (QUEUE, two or more polynomials) or
// k_leaf_tma_c's body; parent indices are the forest's, rebased by the tree's first parent.
constexpr int kForestLeafIter = 2;

template <bool QUEUE>
__global__ void __launch_bounds__(kThreads, QUEUE ? 8 : 6)
    k_fleaf_tma(const ForestTree *__restrict__ trees, const int64_t *__restrict__ off, int S,
                CsfView c, void *const *__restrict__ blk, const int64_t *__restrict__ ctasks,
                uint8_t *__restrict__ keep, uint8_t *__restrict__ flag) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int k = c.k;
  const int64_t *offl = off + (int64_t)(k - 1) * (S + 1);
  const int64_t *offp = off + (int64_t)(k - 2) * (S + 1);
  const int64_t b = blockIdx.x;
  const int t = tree_of(ctasks, S, b);
  const ForestTree &T = trees[t];
  const int64_t o = __ldg(offl + t), n = __ldg(offl + t + 1) - o;
  const int64_t chunk = 2 * (int64_t)kForestLeafIter * kThreads;
  const int64_t first = o + (b - __ldg(ctasks + t)) * chunk;
  const int64_t last = (first + chunk < o + n ? first + chunk : o + n) - 1;
  // the tree's leaf arguments once per CTA in shared memory (indexed by polynomial at run
  // time, which a per-thread copy would keep in local memory)
  __shared__ LeafArgs A;
  const int npoly = T.dev.npoly;
  if (threadIdx.x == 0)
    for (int f = 0; f < npoly; ++f) {
      A.rel[f] = T.dev.rel[f];
      A.in[f] = blk[((int64_t)t * VX_MAXPOLY + f) * VX_KMAX + k - 2];
      A.blk[f] = T.dev.p[f].st[k - 1].blk_in;
      A.len[f] = T.dev.p[f].st[k - 1].maxlen;
    }
  __syncthreads();
  const int64_t poff = __ldg(offp + t);
  if constexpr (QUEUE) {
    __shared__ LeafQueue<kForestLeafIter> Q;
    leaf_q_chunk<kForestLeafIter>(A, npoly, c.lab[k - 1], c.par[k - 1], poff, first, last,
                                  T.ax[k - 1], keep, flag, smem, Q);
  } else {
    leaf_tma_c_chunk(A, npoly, c.lab[k - 1], c.par[k - 1], poff, first, last, 0, T.ax[k - 1],
                     keep, nullptr, nullptr, flag, smem);
  }
}

template <class AR>
int eval_forest_t(const ForestTree *d_trees, const ForestTree *h_trees, const int64_t *d_off,
                  const int64_t *h_off, int S, const CsfView &c, uint8_t *keep, uint8_t *flag,
                  float theta, cudaStream_t s, int64_t *madds) {
  using V = typename AR::V;
  const int k = c.k;
  *madds = 0;
  if (c.N[k - 1] == 0) return VX_OK;
  // blocks of every (tree, polynomial, depth < k-1), node-major, one allocation
  std::vector<void *> tab((size_t)S * VX_MAXPOLY * VX_KMAX, nullptr);
  std::vector<size_t> at(tab.size(), 0);
  size_t total = 0;
  for (int t = 0; t < S; ++t)
    for (int f = 0; f < h_trees[t].dev.npoly; ++f)
      for (int d = 0; d < k; ++d) {
        const int64_t nd = h_off[(int64_t)d * (S + 1) + t + 1] - h_off[(int64_t)d * (S + 1) + t];
        const StageDev &st = h_trees[t].dev.p[f].st[d];
        *madds += nd * (st.blk_in - st.nfib);
        if (d + 1 < k) {
          at[((size_t)t * VX_MAXPOLY + f) * VX_KMAX + d] = total;
          total += ((size_t)nd * st.blk_out * sizeof(V) + 255) & ~(size_t)255;
        }
      }
  void *mem = nullptr, *dtab = nullptr;
  int rc = VX_OK;
  if (total > 0) rc = dmalloc(&mem, total, s);
  if (rc == VX_OK) rc = dmalloc(&dtab, tab.size() * sizeof(void *), s);
  if (rc == VX_OK) {
    for (size_t j = 0; j < tab.size(); ++j) tab[j] = mem ? (char *)mem + at[j] : nullptr;
    // from pageable memory: returns once the table is staged, so `tab` may go
    if (cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(void *), cudaMemcpyHostToDevice,
                        s) != cudaSuccess) {
      set_error("forest block table upload failed");
      rc = VX_ECUDA;
    }
  }
  // warp-task queues: per depth, per tree, chunks of 32 nodes (64 in pairs) x G fibre groups
  std::vector<int64_t> tasks((size_t)k * (S + 1), 0);
  bool pairs[VX_KMAX] = {false};
  int G[VX_KMAX];
  for (int d = 0; d < VX_KMAX; ++d) G[d] = 1;
  for (int d = 0; d < k; ++d) {
    const bool leaf = d + 1 == k;
    pairs[d] = std::is_same<AR, A32C>::value && (leaf || c.N[d] >= kPairNodes);
    const int64_t per = pairs[d] ? 64 : 32;
    int64_t chunks = 0, maxfib = 1;
    for (int t = 0; t < S; ++t) {
      const int64_t nd = h_off[(int64_t)d * (S + 1) + t + 1] - h_off[(int64_t)d * (S + 1) + t];
      chunks += (nd + per - 1) / per;
      for (int f = 0; f < h_trees[t].dev.npoly; ++f)
        maxfib = std::max<int64_t>(maxfib, h_trees[t].dev.p[f].st[d].nfib);
    }
    if (!leaf && chunks > 0) G[d] = (int)std::min<int64_t>(maxfib, std::max<int64_t>(1, ((int64_t)sm_count() * 64 + chunks - 1) / chunks));
    int64_t acc = 0;
    for (int t = 0; t < S; ++t) {
      tasks[(size_t)d * (S + 1) + t] = acc;
      const int64_t nd = h_off[(int64_t)d * (S + 1) + t + 1] - h_off[(int64_t)d * (S + 1) + t];
      acc += (nd + per - 1) / per * G[d];
    }
    tasks[(size_t)d * (S + 1) + S] = acc;
  }
  void *dtasks = nullptr;
  if (rc == VX_OK) rc = dmalloc(&dtasks, tasks.size() * sizeof(int64_t), s);
  if (rc == VX_OK && cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(int64_t),
                                     cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("forest task table upload failed");
    rc = VX_ECUDA;
  }
  auto blocks_of = [](int64_t ntask) {
    int64_t b = (ntask + kWarpsPerBlock - 1) / kWarpsPerBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 32));
  };
  for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
    const int64_t *td = (const int64_t *)dtasks + (size_t)d * (S + 1);
    const unsigned nb = blocks_of(tasks[(size_t)d * (S + 1) + S]);
    if (pairs[d])
      k_fstage<AR, true><<<nb, kThreads, 0, s>>>(d_trees, d_off, S, d, c, (void *const *)dtab, td, G[d]);
    else
      k_fstage<AR, false><<<nb, kThreads, 0, s>>>(d_trees, d_off, S, d, c, (void *const *)dtab, td, G[d]);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("forest stage launch failed");
      rc = VX_ECUDA;
    }
  }
  // certified binary32 leaves with parents: the staged single-system bodies, one CTA per
  // chunk of a tree's leaves, when every tree's staged blocks fit in shared memory
  bool staged_leaf = std::is_same<AR, A32C>::value && k >= 2;
  size_t leaf_smem = 128;
  int maxpoly = 0;
  std::vector<int64_t> ctasks(S + 1, 0);
  if (staged_leaf) {
    const int64_t chunk = 2 * (int64_t)kForestLeafIter * kThreads;
    for (int t = 0; t < S; ++t) {
      size_t need = 128;
      for (int f = 0; f < h_trees[t].dev.npoly; ++f)
        need += (size_t)kLeafParents * h_trees[t].dev.p[f].st[k - 1].blk_in * sizeof(float4);
      leaf_smem = std::max(leaf_smem, need);
      maxpoly = std::max(maxpoly, h_trees[t].dev.npoly);
      const int64_t nt = h_off[(int64_t)(k - 1) * (S + 1) + t + 1] - h_off[(int64_t)(k - 1) * (S + 1) + t];
      ctasks[t + 1] = ctasks[t] + (nt + chunk - 1) / chunk;
    }
    staged_leaf = leaf_smem <= kMaxDynSmem && ctasks[S] <= INT32_MAX;
  }
  void *dctasks = nullptr;
  if (rc == VX_OK && staged_leaf) {
    rc = dmalloc(&dctasks, ctasks.size() * sizeof(int64_t), s);
    if (rc == VX_OK && cudaMemcpyAsync(dctasks, ctasks.data(), ctasks.size() * sizeof(int64_t),
                                       cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("forest leaf task table upload failed");
      rc = VX_ECUDA;
    }
  }
  if (rc == VX_OK && staged_leaf) {
    if (ctasks[S] > 0) {
      const bool queue = maxpoly >= 2;
      cudaError_t e = queue ? cudaFuncSetAttribute(k_fleaf_tma<true>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)leaf_smem)
                            : cudaFuncSetAttribute(k_fleaf_tma<false>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)leaf_smem);
      if (e == cudaSuccess) {
        if (queue)
          k_fleaf_tma<true><<<(unsigned)ctasks[S], kThreads, leaf_smem, s>>>(
              d_trees, d_off, S, c, (void *const *)dtab, (const int64_t *)dctasks, keep, flag);
        else
          k_fleaf_tma<false><<<(unsigned)ctasks[S], kThreads, leaf_smem, s>>>(
              d_trees, d_off, S, c, (void *const *)dtab, (const int64_t *)dctasks, keep, flag);
        note_launch();
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) {
        set_error("forest leaf launch failed: %s", cudaGetErrorString(e));
        rc = VX_ECUDA;
      }
    }
  } else if (rc == VX_OK) {
    const int64_t *tl = (const int64_t *)dtasks + (size_t)(k - 1) * (S + 1);
    const unsigned nb = blocks_of(tasks[(size_t)(k - 1) * (S + 1) + S]);
    if (pairs[k - 1])
      k_fleaf<AR, true><<<nb, kThreads, 0, s>>>(d_trees, d_off, S, c, (void *const *)dtab, tl, keep, flag, theta);
    else
      k_fleaf<AR, false><<<nb, kThreads, 0, s>>>(d_trees, d_off, S, c, (void *const *)dtab, tl, keep, flag, theta);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("forest leaf launch failed");
      rc = VX_ECUDA;
    }
  }
  dfree(dctasks, s);
  dfree(dtasks, s);
  dfree(dtab, s);
  dfree(mem, s);
  return rc;
}

}  // namespace

int eval_forest(int arith, const ForestTree *d_trees, const ForestTree *h_trees,
                const int64_t *d_off, const int64_t *h_off, int S, const CsfView &c,
                uint8_t *keep, uint8_t *flag, float theta, cudaStream_t s, int64_t *madds) {
  switch (arith) {
    case ARITH_F64:
      return eval_forest_t<A64>(d_trees, h_trees, d_off, h_off, S, c, keep, flag, theta, s, madds);
    case ARITH_F32_MIDRAD:
      return eval_forest_t<A32>(d_trees, h_trees, d_off, h_off, S, c, keep, flag, theta, s, madds);
    default:
      return eval_forest_t<A32C>(d_trees, h_trees, d_off, h_off, S, c, keep, flag, theta, s, madds);
  }
}

int eval_level_taylor(const SysDev &tsys, const int8_t (*alpha)[VX_KMAX], int m,
                      const CsfView &c, const LevelGrid &grid, uint8_t *d_keep, int first, int rel,
                      double *d_lo, double *d_hi, uint8_t *d_inc, uint8_t *d_flag, cudaStream_t s,
                      Timer *tm, int64_t *madds) {
  const int k = c.k;
  TaylorLeaf tl{};
  tl.na = tsys.npoly;
  tl.m = m;
  tl.k = k;
  tl.first = first;
  tl.rel = rel;
  tl.lo = d_lo;
  tl.hi = d_hi;
  if (d_inc) {
    tl.c1 = 1;
    tl.inc = d_inc;
    for (int d = 0; d < k; ++d) {
      tl.ei[d] = -1;
      for (int a = 0; a < tsys.npoly; ++a) {
        bool unit = true;
        for (int j = 0; j < k; ++j) unit = unit && alpha[a][j] == (j == d ? 1 : 0);
        if (unit) tl.ei[d] = (int8_t)a;
      }
      if (tl.ei[d] < 0 || m < 2) {
        set_error("C1 on the Taylor form needs order >= 2");
        return VX_EINVAL;
      }
    }
  }
  std::vector<LevelGrid> pg(tsys.npoly, grid);
  for (int a = 0; a < tsys.npoly; ++a) {
    int tot = 0;
    for (int d = 0; d < VX_KMAX; ++d) {
      tl.alpha[a][d] = d < k ? alpha[a][d] : 0;
      tot += tl.alpha[a][d];
    }
    if (tot < m)
      for (int d = 0; d < k; ++d) {
        pg[a].ax[d].point = 1;
        pg[a].ax[d].fexact = 0;
      }
  }
  for (int d = 0; d < k; ++d) tl.r[d] = 0.5 * grid.ax[d].w;  // exact (dyadic widths)
  if (d_flag) {  // certified binary32: every G_a in A32C
    tl.flag = d_flag;
    for (int a = 0; a < tsys.npoly; ++a)
      for (int d = 0; d < k; ++d)
        if (pg[a].ax[d].point) pg[a].ax[d].fexact = grid.ax[d].fexact;
    return eval_level_t<A32C>(tsys, c, grid, nullptr, nullptr, d_keep, nullptr, 0.f, s, tm, madds,
                              KK_STAGE0_F32C, nullptr, 0, pg.data(), &tl);
  }
  return eval_level_t<A64>(tsys, c, grid, nullptr, nullptr, d_keep, nullptr, 0.f, s, tm, madds,
                           KK_STAGE0, nullptr, 0, pg.data(), &tl);
}

int eval_c1_vertex(const SysDev &sys, const CsfView &c, const LevelGrid &grid, uint8_t *d_inc,
                   cudaStream_t s, Timer *tm, int64_t *madds) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  *madds = 0;
  if (n == 0) return VX_OK;
  if (sys.npoly != 1) {
    set_error("C1 is a test for one equation (the system has %d)", sys.npoly);
    return VX_EINVAL;
  }
  double *lo = nullptr, *hi = nullptr;
  uint8_t *scratch = nullptr, *flags = nullptr;
  int rc = dmalloc((void **)&lo, (size_t)n * 8, s);
  if (rc == VX_OK) rc = dmalloc((void **)&hi, (size_t)n * 8, s);
  if (rc == VX_OK) rc = dmalloc((void **)&scratch, (size_t)n, s);
  if (rc == VX_OK) rc = dmalloc((void **)&flags, (size_t)n, s);
  for (int v = 0; v < (1 << k) && rc == VX_OK; ++v) {
    LevelGrid g = grid;
    for (int d = 0; d < k; ++d) {
      g.ax[d].point = ((v >> (k - 1 - d)) & 1) ? 3 : 2;
      g.ax[d].fexact = 0;
    }
    int64_t w = 0;
    rc = eval_level_t<A64>(sys, c, g, lo, hi, scratch, nullptr, 0.f, s, tm, &w, KK_STAGE0);
    *madds += w;
    if (rc == VX_OK) {
      k_c1_fold<<<leaf_grid(n), kThreads, 0, s>>>(lo, hi, n, flags, v == 0);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) {
        set_error("C1 fold launch failed");
        rc = VX_ECUDA;
      }
    }
  }
  if (rc == VX_OK) {
    k_c1_final<<<leaf_grid(n), kThreads, 0, s>>>(flags, n, d_inc);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("C1 launch failed");
      rc = VX_ECUDA;
    }
  }
  dfree(lo, s);
  dfree(hi, s);
  dfree(scratch, s);
  dfree(flags, s);
  return rc;
}

int set_autotune(int mode, const char *path) {
  Tuner &T = tuner();
  std::lock_guard<std::mutex> g(T.mu);
  T.mode = mode < 0 ? 0 : mode;
  T.path = path ? path : "";
  if (!T.path.empty()) {
    if (FILE *fp = std::fopen(T.path.c_str(), "r")) {
      unsigned long long key = 0;
      int v = 0;
      while (std::fscanf(fp, "%llx %d", &key, &v) == 2) T.best[(uint64_t)key] = v;
      std::fclose(fp);
    }
  }
  return VX_OK;
}

int autotune_entries() {
  Tuner &T = tuner();
  std::lock_guard<std::mutex> g(T.mu);
  return (int)T.best.size();
}

void autotune_clear() {
  Tuner &T = tuner();
  std::lock_guard<std::mutex> g(T.mu);
  T.best.clear();
}

int set_wait_polls(int64_t polls) {
  const uint32_t v = polls < 0 ? kWaitPolls : (polls > 0xffffffffll ? 0xffffffffu : (uint32_t)polls);
  VX_CUDA(cudaMemcpyToSymbol(g_vx_wait_polls, &v, sizeof(v)));
  return VX_OK;
}

int *status_word() {
  static thread_local int *p = nullptr;
  if (!p && cudaHostAlloc((void **)&p, sizeof(int), cudaHostAllocDefault) != cudaSuccess) p = nullptr;
  return p;
}

int queue_device_status(cudaStream_t s, int *h_pinned) {
  VX_CUDA(cudaMemcpyFromSymbolAsync(h_pinned, g_vx_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  return VX_OK;
}

int take_device_status(cudaStream_t s, int *status) {
  int v = 0;
  VX_CUDA(cudaMemcpyFromSymbolAsync(&v, g_vx_status, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
  VX_CUDA(cudaStreamSynchronize(s));
  if (v) {
    const int zero = 0;
    VX_CUDA(cudaMemcpyToSymbolAsync(g_vx_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
    VX_CUDA(cudaStreamSynchronize(s));
  }
  *status = v;
  return VX_OK;
}

// ---------------------------------------------------------------------------------------
// The float-pair tier, run on the boxes of the certified binary32 path's error band before
// binary64.  Each interval end is a pair (h, l) of binary32 numbers standing for h + l with
// |l| <= ulp(h) / 2 (about 48 bits), an interval stored as (lo_h, lo_l, -hi_h, -hi_l), and a
// bound E on |lo_pair - lo*| + |lo64 - lo*| (the same for hi), lo* the exact interval Horner
// value with the binary64 coefficients and lo64 what the binary64 path computes.
//
// One step J*Y + C on Y = [yl, yh] >= 0 (a box with x <= 0 runs Horner in y = -x on the
// coefficients (-1)^a C_a, as the certified binary32 leaves do), per end, m the end of Y at
// which that end's product is smallest (yl where the end is >= 0, whose sign is its h's):
//   ph = RN(h m), pe = FMA(h, m, -ph) (the product's exact error), pl = RN(l m + pe);
//   (sh, se) = TwoSum(ph, C_h); u = RN(se + RN(pl + C_l)); (rh, rl) = TwoSum(sh, u).
// The min over the ends of Y of J's end times y is xmax-Lipschitz in that end, the roundings
// (pl, RN(pl + C_l), u) stay below 2^-45 (|J| yh + |C|) together, and binary64 rounds its
// product and sum downward (< 2^-52 of magnitudes at most |J| yh + |C| + the distances), so
//   E' = RU(E_J xp + RU(2^-43 T + E_C (1 + 2^-40))) + 2^-145,
//   T = max|ends of J| yh + max|ends of C|,  xp = RU(yh (1 + 2^-40)),
// bounds the new distance (2^-145 covers the absolute errors below the normal range).  A
// decision compares the exact sum h + l (in binary64) with E.  Boxes straddling 0 and grids
// whose box ends are not binary32 numbers are left to binary64 (E infinite).
// ---------------------------------------------------------------------------------------
namespace {

struct PairX {
  float yl, yh, xp;
  bool neg;  // the box is x <= 0: Horner runs in y = -x
  bool ok;   // the box does not straddle 0
};

__device__ __forceinline__ PairX pair_box(const AxisGrid &g, int32_t t) {
  PairX x;
  const float l = __fmaf_rn((float)t, g.fw, g.flo), h = __fmaf_rn((float)t + 1.0f, g.fw, g.flo);
  x.ok = l >= 0.f || h <= 0.f;
  x.neg = !(l >= 0.f);
  x.yl = x.neg ? -h : l;
  x.yh = x.neg ? -l : h;
  x.xp = __fmaf_ru(x.yh, 0x1p-40f, x.yh);
  return x;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// the lower end of (jh + jl) * [yl, yh] + (ch + cl), yl >= 0
__device__ __forceinline__ void pair_end(float jh, float jl, float yl, float yh, float ch,
                                         float cl, float &rh, float &rl) {
  const float m = jh >= 0.f ? yl : yh;
  const float ph = __fmul_rn(jh, m);
  const float pe = __fmaf_rn(jh, m, -ph);
  const float pl = __fmaf_rn(jl, m, pe);
  float sh, se;
  two_sum(ph, ch, sh, se);
  const float u = __fadd_rn(se, __fadd_rn(pl, cl));
  two_sum(sh, u, rh, rl);
}

__device__ __forceinline__ float4 pair_negated(const float4 c) {
  return make_float4(c.z, c.w, c.x, c.y);
}

__device__ __forceinline__ void pair_step(float4 &j, float &ej, const float4 &c, float ec,
                                          const PairX &x) {
  const float MJ = fmaxf(fabsf(j.x), fabsf(j.z)), MC = fmaxf(fabsf(c.x), fabsf(c.z));
  float4 r;
  pair_end(j.x, j.y, x.yl, x.yh, c.x, c.y, r.x, r.y);
  pair_end(j.z, j.w, x.yl, x.yh, c.z, c.w, r.z, r.w);
  const float T = __fmaf_ru(MJ, x.yh, MC);
  float e = __fmaf_ru(ec, 0x1p-40f, ec);
  e = __fmaf_ru(0x1p-43f, T, e);
  e = __fmaf_ru(ej, x.xp, e);
  ej = __fadd_ru(e, 0x1p-145f);
  j = r;
}

// Algorithm 1 on one fibre (entry a at vb[(rowoff[a] + f) estride], its bound in eb; with
// fiboff non-null at vb[fiboff[f] + a], the fibre-major block), Horner in y = -x with odd
// coefficients negated when the box is x <= 0 (the result is J itself).
__device__ __forceinline__ void pair_horner(const float4 *__restrict__ vb,
                                            const float *__restrict__ eb, int64_t estride,
                                            const int32_t *__restrict__ rowoff, int f, int L,
                                            const PairX &x, float4 &J, float &E,
                                            const int32_t *__restrict__ fiboff = nullptr) {
  const int64_t fo = fiboff ? (int64_t)__ldg(fiboff + f) : 0;
  auto at = [&](int a) {
    return fiboff ? fo + a : (int64_t)(__ldg(rowoff + a) + f) * estride;
  };
  int64_t o = at(L - 1);
  const float4 top = vb[o];
  E = eb[o];
  J = (x.neg && ((L - 1) & 1)) ? pair_negated(top) : top;
  for (int a = L - 2; a >= 0; --a) {
    o = at(a);
    float4 c = vb[o];
    const float ec = eb[o];
    if (x.neg && (a & 1)) c = pair_negated(c);
    pair_step(J, E, c, ec, x);
  }
}

// 0: the binary64 path surely drops the box for this relation, 1: surely not, 2: unknown
__device__ __forceinline__ int pair_classify(const float4 &J, float E, int rel) {
  const double lo = (double)J.x + (double)J.y, nhi = (double)J.z + (double)J.w;  // exact
  const double e = (double)E;
  const bool fin = E < INFINITY && isfinite(lo) && isfinite(nhi);
  if (!fin) return 2;
  // lo64 lies in [lo - e, lo + e], -hi64 in [nhi - e, nhi + e]
  const double lo_dn = __dadd_rd(lo, -e), lo_up = __dadd_ru(lo, e);
  const double nh_dn = __dadd_rd(nhi, -e), nh_up = __dadd_ru(nhi, e);
  switch (rel) {
    case VX_LE: return lo_dn > 0.0 ? 0 : (lo_up <= 0.0 ? 1 : 2);    // drop iff lo64 > 0
    case VX_GE: return nh_dn > 0.0 ? 0 : (nh_up <= 0.0 ? 1 : 2);    // drop iff hi64 < 0
    case VX_LT: return lo_dn >= 0.0 ? 0 : (lo_up < 0.0 ? 1 : 2);    // drop iff lo64 >= 0
    case VX_GT: return nh_dn >= 0.0 ? 0 : (nh_up < 0.0 ? 1 : 2);    // drop iff hi64 <= 0
    default:
      if (lo_dn > 0.0 || nh_dn > 0.0) return 0;
      if (lo_up <= 0.0 && nh_up <= 0.0) return 1;
      return 2;
  }
}

// Stage d on every depth-d node of the tier's tree: thread = (fibre f, node), consecutive
// threads on consecutive nodes of one fibre.  Input entry e of parent p at
// in[e * in_estride + p * in_nstride] (the coefficients: 1, 0); output entry-major.
__global__ void __launch_bounds__(256)
    k_stage_pair(const StageDev st, const int32_t *__restrict__ lab,
                 const int32_t *__restrict__ par, const float4 *__restrict__ in_v,
                 const float *__restrict__ in_e, int64_t in_estride, int64_t in_nstride,
                 float4 *__restrict__ out_v, float *__restrict__ out_e, int64_t nnodes,
                 AxisGrid g, bool fm) {
  const int64_t total = nnodes * st.nfib;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; it < total; it += stride) {
    const int f = (int)(it / nnodes);
    const int64_t node = it - (int64_t)f * nnodes;
    const PairX x = pair_box(g, __ldg(lab + node));
    const int64_t p = par ? (int64_t)__ldg(par + node) : 0;
    float4 J = make_float4(0.f, 0.f, 0.f, 0.f);
    float E = INFINITY;
    if (x.ok)
      pair_horner(in_v + p * in_nstride, in_e + p * in_nstride, in_estride, st.rowoff, f,
                  __ldg(st.fiblen + f), x, J, E, fm ? st.fiboff : nullptr);
    const int64_t o = (int64_t)__ldg(st.outpos + f) * nnodes + node;
    out_v[o] = J;
    out_e[o] = E;
  }
}

struct PairLeafArgs {
  const float4 *in_v[VX_MAXPOLY];  // parent blocks, entry-major (the coefficients when k == 1)
  const float *in_e[VX_MAXPOLY];
  const int32_t *rowoff[VX_MAXPOLY];
  int32_t len[VX_MAXPOLY];
  int8_t rel[VX_MAXPOLY];
};

__global__ void __launch_bounds__(256)
    k_leaf_pair(PairLeafArgs A, int npoly, const int32_t *__restrict__ lab,
                const int32_t *__restrict__ par, int64_t nleaves, int64_t nparents, AxisGrid g,
                uint8_t *__restrict__ keep, uint8_t *__restrict__ flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nleaves; i += stride) {
    const PairX x = pair_box(g, __ldg(lab + i));
    bool ex = false, am = !x.ok;
    if (x.ok) {
      const int64_t p = par ? (int64_t)__ldg(par + i) : 0;
      const int64_t es = par ? nparents : 1;
      for (int f = 0; f < npoly && !ex; ++f) {
        float4 J;
        float E;
        pair_horner(A.in_v[f] + (par ? p : 0), A.in_e[f] + (par ? p : 0), es, A.rowoff[f], 0,
                    A.len[f], x, J, E);
        const int r = pair_classify(J, E, A.rel[f]);
        ex = ex || r == 0;
        am = am || r == 2;
      }
    }
    keep[i] = ex ? 0 : 1;
    flag[i] = (!ex && am) ? 1 : 0;
  }
}

}  // namespace

int eval_level_pair(const SysDev &sys, const CsfView &c, const LevelGrid &grid, uint8_t *d_keep,
                    uint8_t *d_flag, cudaStream_t s, Timer *tm, int64_t *madds_out) {
  const int k = sys.k;
  const int64_t nleaves = c.N[k - 1];
  *madds_out = 0;
  if (nleaves == 0) return VX_OK;
  bool exact = true;
  for (int d = 0; d < k; ++d)
    exact = exact && grid.ax[d].fexact && !grid.ax[d].point && !grid.ax[d].xlo;
  if (!exact) {  // box ends that are not binary32 numbers: everything goes to binary64
    VX_CUDA(cudaMemsetAsync(d_keep, 1, (size_t)nleaves, s));
    VX_CUDA(cudaMemsetAsync(d_flag, 1, (size_t)nleaves, s));
    return VX_OK;
  }
  float4 *val[VX_MAXPOLY][VX_KMAX] = {{nullptr}};
  float *err[VX_MAXPOLY][VX_KMAX] = {{nullptr}};
  int rc = VX_OK;
  int64_t madds = 0;
  auto grid_of = [](int64_t items) {
    int64_t b = (items + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 16;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, cap));
  };
  for (int f = 0; f < sys.npoly && rc == VX_OK; ++f) {
    for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
      const StageDev &st = sys.p[f].st[d];
      const int64_t n = c.N[d] * st.blk_out;
      rc = dmalloc((void **)&val[f][d], (size_t)std::max<int64_t>(n, 1) * sizeof(float4), s);
      if (rc == VX_OK) rc = dmalloc((void **)&err[f][d], (size_t)std::max<int64_t>(n, 1) * sizeof(float), s);
      if (rc != VX_OK) break;
      const int64_t w = c.N[d] * (st.blk_in - st.nfib);
      madds += w;
      if (tm && tm->on) rc = tm->begin(d == 0 ? KK_STAGE0_PAIR : KK_STAGEJ_PAIR, w);
      if (rc != VX_OK) break;
      // stage 0 from the fibre-major copies of the coefficients (consecutive loads along a
      // fibre)
      const bool fm0 = d == 0 && sys.p[f].cp_fm && sys.p[f].ep_fm;
      const float4 *in_v = d == 0 ? (fm0 ? sys.p[f].cp_fm : sys.p[f].cp) : val[f][d - 1];
      const float *in_e = d == 0 ? (fm0 ? sys.p[f].ep_fm : sys.p[f].ep) : err[f][d - 1];
      k_stage_pair<<<grid_of(c.N[d] * st.nfib), 256, 0, s>>>(
          st, c.lab[d], d == 0 ? nullptr : c.par[d], in_v, in_e, d == 0 ? 1 : c.N[d - 1],
          d == 0 ? 0 : 1, val[f][d], err[f][d], c.N[d], grid.ax[d], fm0);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) {
        set_error("float-pair stage launch failed");
        rc = VX_ECUDA;
      }
      if (rc == VX_OK && tm && tm->on) rc = tm->end();
    }
  }
  if (rc == VX_OK) {
    PairLeafArgs A{};
    int64_t wl = 0;
    for (int f = 0; f < sys.npoly; ++f) {
      const StageDev &st = sys.p[f].st[k - 1];
      A.in_v[f] = k == 1 ? sys.p[f].cp : val[f][k - 2];
      A.in_e[f] = k == 1 ? sys.p[f].ep : err[f][k - 2];
      A.rowoff[f] = st.rowoff;
      A.len[f] = st.maxlen;
      A.rel[f] = sys.rel[f];
      wl += nleaves * (st.blk_in - 1);
    }
    madds += wl;
    if (tm && tm->on) rc = tm->begin(KK_LEAF_PAIR, wl);
    if (rc == VX_OK) {
      k_leaf_pair<<<grid_of(nleaves), 256, 0, s>>>(A, sys.npoly, c.lab[k - 1],
                                                   k == 1 ? nullptr : c.par[k - 1], nleaves,
                                                   k == 1 ? 0 : c.N[k - 2], grid.ax[k - 1],
                                                   d_keep, d_flag);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) {
        set_error("float-pair leaf launch failed");
        rc = VX_ECUDA;
      }
    }
    if (rc == VX_OK && tm && tm->on) rc = tm->end();
  }
  for (int f = 0; f < sys.npoly; ++f)
    for (int d = 0; d + 1 < k; ++d) {
      dfree(val[f][d], s);
      dfree(err[f][d], s);
    }
  *madds_out = madds;
  return rc;
}

// ---------------------------------------------------------------------------------------
// Level evaluation without allocating: the partial-evaluation blocks live in a fixed array of
// device memory that belongs to the library (every device that loads the library holds it
// until the process exits).  The kernels are the ones above; only host code needs the array's
// device address, which cudaGetSymbolAddress gives once per device.
// ---------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_vx_static_scratch[VX_STATIC_SCRATCH_BYTES];

// The array's device address per device ordinal, looked up by the first call on that device
// (with it current) and kept; the lock makes concurrent first calls from several host threads
// safe.  The address belongs to the device's context: a cudaDeviceReset on that device ends it.
static std::mutex g_static_scratch_mu;
static void *g_static_scratch_addr[64] = {nullptr};

int static_scratch_address(void **addr) {
  int dev = 0;
  VX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("device ordinal %d is outside the supported range", dev);
    return VX_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_scratch_mu);
  if (!g_static_scratch_addr[dev]) {
    void *p = nullptr;
    VX_CUDA(cudaGetSymbolAddress(&p, g_vx_static_scratch));
    g_static_scratch_addr[dev] = p;
  }
  *addr = g_static_scratch_addr[dev];
  return VX_OK;
}

int eval_level_static(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, int arith,
                      double *d_lo, double *d_hi, uint8_t *d_keep, cudaStream_t s) {
  void *scratch = nullptr;
  VX_CHECK(static_scratch_address(&scratch));
  if (arith == ARITH_F64)
    return eval_level_t<A64>(sys, csf, grid, d_lo, d_hi, d_keep, nullptr, 0.f, s, nullptr,
                             nullptr, KK_STAGE0, scratch, VX_STATIC_SCRATCH_BYTES);
  return eval_level_t<A32>(sys, csf, grid, d_lo, d_hi, d_keep, nullptr, 0.f, s, nullptr, nullptr,
                           KK_STAGE0_F32, scratch, VX_STATIC_SCRATCH_BYTES);
}

int eval_level_raw(const SysDev &sys, const CsfView &csf, const LevelGrid &grid, int arith,
                   double *d_lo, double *d_hi, uint8_t *d_keep, uint8_t *d_flag, float theta,
                   cudaStream_t s, Timer *tm, int64_t *madds_out) {
  switch (arith) {
    case ARITH_F64:
      return eval_level_t<A64>(sys, csf, grid, d_lo, d_hi, d_keep, d_flag, theta, s, tm,
                               madds_out, KK_STAGE0);
    case ARITH_F32_MIDRAD:
      return eval_level_t<A32>(sys, csf, grid, d_lo, d_hi, d_keep, d_flag, theta, s, tm,
                               madds_out, KK_STAGE0_F32);
    default:
      return eval_level_t<A32C>(sys, csf, grid, d_lo, d_hi, d_keep, d_flag, theta, s, tm,
                                madds_out, KK_STAGE0_F32C);
  }
}

}  // namespace vx
