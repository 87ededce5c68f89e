// vx_dense.cu -- a full-grid level of a dense trivariate system on the tensor cores.
//
// Property 1 (Sec. 1) writes a polynomial on a tensor grid as mode-by-mode contractions of its
// coefficient tensor C[a1][a2][a3] with the Vandermonde matrices of the grid.  On every box
// of the level (N = 2^level boxes per axis, centre c, half-width r) this file computes a
// midpoint-radius enclosure of each polynomial in that form, one contraction per variable:
//
//   mode j:  mid_out[..] = sum_a mid_in[a] c^a
//            rad_out[..] = sum_a |mid_in[a]| ((|c|+r)^a - |c|^a)  +  rad_in[a] (|c|+r)^a
//
// (for x = c + e, |e| <= r: |(c+e)^a - c^a| <= (|c|+r)^a - |c|^a and |(c+e)^a| <= (|c|+r)^a, so
// every value of the polynomial on the box lies within rad_out of mid_out).  By induction over
// Horner's steps this enclosure contains the midpoint-radius Horner enclosure, which contains
// the endpoint (inf-sup) interval Horner enclosure of Algorithm 1: a box it excludes is
// excluded by criterion C0 of Sec. 3.2 as well, so its kept set is a superset of the exact
// kept set and serves as a prefilter (the survivors are then decided exactly).
//
// Each contraction is a pair of TF32 GEMMs on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory): one for the midpoints and one, over the concatenated inner
// dimension [|mid_in| rad_in] x [(|c|+r)^a - |c|^a ; (|c|+r)^a], for the radii.  The inputs are
// rounded to TF32 before they are stored, so the products are exact in binary32; the rounding
// of the Vandermonde entries and of the accumulation is charged to the radius through the
// factor matrix ((|c|+r)^a - |c|^a + kappa |c|^a, kappa = 2^-10, every factor rounded up) and
// a relative factor 1 + 2^-12 on each accumulated radius.  The epilogue of modes 1 and 2 rounds
// the midpoints to TF32 (adding the rounding to the radius) and writes them straight into the
// next mode's operand layout; mode 3's epilogue writes one bit per box (1 = may hold a zero).
//
// Operand layout (both operands K-major, no swizzle): a panel of 128 (A) or NT (B) rows is a
// sequence of k-steps of 8 columns; a k-step holds the rows in groups of 8, each group two 8x16
// byte core matrices (columns 0-3, then 4-7).  A k-step of a panel is one contiguous block
// (4 KB for A), so a stage of the pipeline is a few 1-D TMA bulk copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "vx_internal.cuh"
#include "vx_ptx.cuh"

namespace vx {
namespace {

constexpr int kStages = 3;  // pipeline depth
constexpr int kG = 4;       // k-steps (of 8) per stage
constexpr int kAStep = 4096;  // bytes of one A k-step (128 rows x 8 x 4 B)
// Charged to the radius for the binary32/TF32 arithmetic of the contractions: kKappa |c|^a per
// term for the midpoint's error (TF32 rounding of a Vandermonde entry, below 2^-10.99 of it,
// plus the accumulation, assumed below 2^-22 of the running sum of |products| per addition:
// at most 2^-14 of the sum over <= 256 terms), and a relative kRadRel on each accumulated
// radius (accumulation of <= 512 nonnegative terms, at most 2^-13).
constexpr float kKappa = 0x1p-10f;
constexpr float kRadRel = 0x1p-12f;

// Nonzero after a bounded wait gave up in a tensor-core kernel (read by take_dense_status).
__device__ int g_vx_dense_status = 0;
// Polls of a pipeline wait (a stage's copies, a stage's MMAs) before giving up (settable for
// tests); the waits that drain work already issued (copies in flight, the MMAs of the tile)
// before the block frees its tensor memory and exits use the fixed kDrainPolls.
constexpr uint32_t kDenseWaitPolls = 1u << 24;
constexpr uint32_t kDrainPolls = 1u << 24;
__device__ uint32_t g_vx_dense_wait_polls = kDenseWaitPolls;

__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(&g_vx_dense_status, 1);
  return false;
}

// binary32 -> TF32 (10 explicit mantissa bits): nearest, and upward for values >= 0
__host__ __device__ __forceinline__ uint32_t f2u(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  return u;
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
  float x;
  memcpy(&x, &u, 4);
  return x;
}
__host__ __device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = f2u(x);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;
  return u2f(u);
}
__host__ __device__ __forceinline__ float tf32_ru_pos(float x) {
  uint32_t u = f2u(x);
  if ((u & 0x7F800000u) != 0x7F800000u && (u & 0x1FFFu)) u = (u | 0x1FFFu) + 1u;
  return u2f(u);
}

// element offset of (row, k) in an A-layout operand (panels of 128 rows, nk k-steps each)
__host__ __device__ __forceinline__ int64_t a_off(int64_t row, int k, int nk) {
  const int64_t tile = row >> 7;
  const int r = (int)(row & 127);
  return ((tile * nk + (k >> 3)) << 10) + ((r >> 3) << 6) + (((k & 7) >> 2) << 5) +
         ((r & 7) << 2) + (k & 3);
}
// ... and in a B-layout operand (panels of NT rows)
__host__ __device__ __forceinline__ int64_t b_off(int64_t row, int k, int nk, int NT) {
  const int64_t tile = row / NT;
  const int r = (int)(row - tile * NT);
  return (tile * nk + (k >> 3)) * (int64_t)(NT * 8) + ((r >> 3) << 6) + (((k & 7) >> 2) << 5) +
         ((r & 7) << 2) + (k & 3);
}

struct TcOperand {
  const float *p;
  int64_t tile_stride;   // floats between consecutive M (or N) panels
  int64_t batch_stride;  // floats between batches (0: shared by all batches)
};

enum Epi { EPI_NEXT_B = 1, EPI_NEXT_A = 2, EPI_BITS = 3, EPI_VALUES = 4 };

struct TcArgs {
  TcOperand A, Ar, B, Br;  // midpoint and radius operands
  int nk, nkr;             // k-steps of the midpoint and of the radius product
  int NT;                  // N of a tile (multiple of 16, <= 256)
  int mtiles, ntiles;
  int64_t batches;
  uint32_t idesc;
  // epilogue
  int64_t N;             // boxes per axis
  int D3p1;              // mode 1: (degree in x3) + 1, to split a column into (a2, a3)
  int64_t ncols;         // mode 1: valid columns (D2+1)(D3+1)
  int nk_next, Kp_next;  // next operand: k-steps of its midpoint panel, padded inner size
  int NT_next;           // mode 1: rows per panel of the next B operand
  float *o_mid, *o_rad;  // next operand (midpoints; [|mid| rad])
  int64_t o_mid_bstride, o_rad_bstride;
  uint32_t *mask;        // mode 3
  int first;             // mode 3: the first polynomial writes, the others AND
  float *v_mid, *v_rad;  // mode 3 values
};

__device__ __forceinline__ float rad_acc_out(float racc) {
  return __fadd_ru(__fmul_ru(racc, 1.0f + kRadRel), 0x1p-100f);
}

template <int EPI>
__device__ __forceinline__ void epilogue(const TcArgs &a, uint32_t tmem, uint32_t radc, int mt,
                                         int nt, int64_t b) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)mt * 128 + warp * 32 + lane;
  const uint32_t lanebase = (uint32_t)(warp * 32) << 16;
  uint32_t word = 0;
  for (int c0 = 0; c0 < a.NT; c0 += 16) {
    float m[16], r[16];
    tmem_ld16(tmem + lanebase + (uint32_t)c0, m);
    tmem_ld16(tmem + lanebase + radc + (uint32_t)c0, r);
    tmem_ld_wait();
    if (EPI == EPI_NEXT_B) {  // mode 1: row = t1, column j = a2 (D3+1) + a3
      if (row < a.N) {
        float *om = a.o_mid + row * a.o_mid_bstride, *orr = a.o_rad + row * a.o_rad_bstride;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int64_t j = (int64_t)nt * a.NT + c0 + i;
          if (j < a.ncols) {
            const int a2 = (int)(j / a.D3p1), a3 = (int)(j - (int64_t)a2 * a.D3p1);
            const float ms = tf32_rn(m[i]);
            const float rs = tf32_ru_pos(__fadd_ru(rad_acc_out(r[i]), fabsf(m[i] - ms)));
            om[b_off(a3, a2, a.nk_next, a.NT_next)] = ms;
            orr[b_off(a3, a2, 2 * a.nk_next, a.NT_next)] = fabsf(ms);
            orr[b_off(a3, a.Kp_next + a2, 2 * a.nk_next, a.NT_next)] = rs;
          }
        }
      }
    } else if (EPI == EPI_NEXT_A) {  // mode 2: batch = t1, row = t2, column = a3
      if (row < a.N) {
        const int64_t mrow = b * a.N + row;
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          const int a3 = c0 + q;
          if (a3 < a.Kp_next) {
            float4 vm, va, vr;
            float *pm = &vm.x, *pa = &va.x, *pr = &vr.x;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float ms = tf32_rn(m[q + i]);
              pm[i] = ms;
              pa[i] = fabsf(ms);
              pr[i] = tf32_ru_pos(__fadd_ru(rad_acc_out(r[q + i]), fabsf(m[q + i] - ms)));
            }
            *reinterpret_cast<float4 *>(a.o_mid + a_off(mrow, a3, a.nk_next)) = vm;
            *reinterpret_cast<float4 *>(a.o_rad + a_off(mrow, a3, 2 * a.nk_next)) = va;
            *reinterpret_cast<float4 *>(a.o_rad + a_off(mrow, a.Kp_next + a3, 2 * a.nk_next)) = vr;
          }
        }
      }
    } else if (EPI == EPI_BITS) {  // mode 3: row = (t1, t2), column = t3
      uint32_t bits = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) bits |= (fabsf(m[i]) > rad_acc_out(r[i]) ? 0u : 1u) << i;
      word |= bits << (c0 & 16);
      const int64_t t3 = (int64_t)nt * a.NT + (c0 & ~31);
      if (c0 & 16) {  // a full word: columns t3 .. t3+31
        if (t3 < a.N) {
          uint32_t *w = a.mask + row * (a.N >> 5) + (t3 >> 5);
          *w = a.first ? word : (*w & word);
        }
        word = 0;
      }
    } else {  // EPI_VALUES
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int64_t t3 = (int64_t)nt * a.NT + c0 + i;
        if (t3 < a.N) {
          a.v_mid[row * a.N + t3] = m[i];
          a.v_rad[row * a.N + t3] = rad_acc_out(r[i]);
        }
      }
    }
  }
}

// One 128 x NT output tile of a mode: D_mid = A B^T over nk k-steps and D_rad = Ar Br^T over
// nkr k-steps, both in tensor memory.  Thread 0 streams the k-steps into a kStages-deep ring of
// shared-memory stages (TMA bulk copies), thread 32 issues the MMAs (tcgen05.commit frees a
// stage once its MMAs have read it), and the four warps read the accumulators back (warp w:
// rows 32w..32w+31) for the epilogue.  Every wait is bounded; a wait that gives up sets
// g_vx_dense_status, the tile's outputs are skipped, and TMEM is freed once the MMAs issued
// so far have completed.
template <int EPI>
__global__ void __launch_bounds__(128, 1) k_tc_mode(const TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const uint32_t bstep = (uint32_t)a.NT * 32;  // bytes of one B k-step
  unsigned char *sA = smem;
  unsigned char *sB = smem + kStages * kG * kAStep;
  uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * kG * bstep);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *slot = reinterpret_cast<uint32_t *>(done + 1);
  int *fail = reinterpret_cast<int *>(slot + 1);
  const int warp = threadIdx.x >> 5;

  int64_t bid = blockIdx.x;
  const int nt = (int)(bid % a.ntiles);
  bid /= a.ntiles;
  const int mt = (int)(bid % a.mtiles);
  const int64_t b = bid / a.mtiles;
  const uint32_t ncols = a.NT > 128 ? 512u : 256u, radc = ncols / 2;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *fail = 0;
  }
  if (warp == 0) tmem_alloc(slot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  const int nsteps = a.nk + a.nkr;
  const int nst = (nsteps + kG - 1) / kG;
  if (threadIdx.x == 0) {  // producer
    const float *pa = a.A.p + b * a.A.batch_stride + (int64_t)mt * a.A.tile_stride;
    const float *par = a.Ar.p + b * a.Ar.batch_stride + (int64_t)mt * a.Ar.tile_stride;
    const float *pb = a.B.p + b * a.B.batch_stride + (int64_t)nt * a.B.tile_stride;
    const float *pbr = a.Br.p + b * a.Br.batch_stride + (int64_t)nt * a.Br.tile_stride;
    int it = 0;
    for (; it < nst; ++it) {
      const int st = it % kStages;
      if (it >= kStages && !wait_bounded(&empty[st], ((it / kStages) - 1) & 1, g_vx_dense_wait_polls)) {
        *fail = 1;
        break;
      }
      const int s0 = it * kG, n = min(kG, nsteps - s0);
      mbar_arrive_expect_tx(&full[st], (uint32_t)n * (kAStep + bstep));
      for (int j = 0; j < n; ++j) {
        const int s = s0 + j;
        const float *srcA = s < a.nk ? pa + (int64_t)s * 1024 : par + (int64_t)(s - a.nk) * 1024;
        const float *srcB = s < a.nk ? pb + (int64_t)s * a.NT * 8 : pbr + (int64_t)(s - a.nk) * a.NT * 8;
        bulk_copy_g2s(sA + (st * kG + j) * kAStep, srcA, kAStep, &full[st]);
        bulk_copy_g2s(sB + (st * kG + j) * bstep, srcB, bstep, &full[st]);
      }
    }
    // copies still in flight land before the block exits (bounded)
    for (int q = std::max(0, it - kStages); q < it; ++q)
      if (!wait_bounded(&full[q % kStages], (q / kStages) & 1, kDrainPolls)) break;
  } else if (threadIdx.x == 32) {  // MMA issuer
    for (int it = 0; it < nst; ++it) {
      const int st = it % kStages;
      if (*(volatile int *)fail || !wait_bounded(&full[st], (it / kStages) & 1, g_vx_dense_wait_polls)) {
        *fail = 1;
        break;
      }
      tc_fence_after();
      const int s0 = it * kG, n = min(kG, nsteps - s0);
      for (int j = 0; j < n; ++j) {
        const int s = s0 + j;
        const uint64_t ad = smem_desc(smem_u32(sA + (st * kG + j) * kAStep), 128, 256);
        const uint64_t bd = smem_desc(smem_u32(sB + (st * kG + j) * bstep), 128, 256);
        if (s < a.nk)
          mma_tf32(tmem, ad, bd, a.idesc, s > 0 ? 1u : 0u);
        else
          mma_tf32(tmem + radc, ad, bd, a.idesc, s > a.nk ? 1u : 0u);
      }
      mma_commit(&empty[st]);
    }
    mma_commit(done);  // every MMA issued above, including after a failure
  }
  __syncwarp();
  const bool ok = wait_bounded(done, 0, kDrainPolls);
  tc_fence_after();
  __syncthreads();
  if (ok && !*(volatile int *)fail) epilogue<EPI>(a, tmem, radc, mt, nt, b);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, ncols);
}

// ---- factor matrices of one axis -----------------------------------------------------------
// x^a for x >= 0 with every product rounded down (up): a lower (upper) bound of the power
__device__ double pow_dir(double x, int e, bool up) {
  double r = 1.0, p = x;
  while (e) {
    if (e & 1) r = up ? __dmul_ru(r, p) : __dmul_rd(r, p);
    e >>= 1;
    if (e) p = up ? __dmul_ru(p, p) : __dmul_rd(p, p);
  }
  return r;
}
__device__ double pow_rn(double x, int e) {
  double r = 1.0, p = x;
  while (e) {
    if (e & 1) r *= p;
    e >>= 1;
    if (e) p *= p;
  }
  return r;
}

enum Factor { F_VAND = 0, F_DIFF = 1, F_POW = 2 };

struct FactorArgs {
  double lo, w;  // grid of the axis: box t = [lo + t w, lo + (t+1) w]
  int64_t N;     // boxes (rows >= N are zero)
  int64_t rows;  // rows written (N rounded up to the panel)
  int D, Kp;     // entries a <= D are nonzero, a < Kp written
  int kind;      // F_VAND: c^a (nearest), F_DIFF: (|c|+r)^a - |c|^a + kappa |c|^a (+ extra
                 // (|c|+r)^a), upward; F_POW: (|c|+r)^a, upward
  double extra;  // F_DIFF: coefficient of the added (|c|+r)^a term
  float *out;
  int layout_b;  // 0: A layout, 1: B layout with NT rows per panel
  int NT, nk, koff;  // panel: nk k-steps; entries go to k = koff + a
};

__global__ void k_factors(FactorArgs f) {
  const int64_t n = f.rows * f.Kp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / f.Kp;
    const int e = (int)(i - t * f.Kp);
    float v = 0.f;
    if (t < f.N && e <= f.D) {
      const double l = f.lo + (double)t * f.w, h = f.lo + (double)(t + 1) * f.w;
      const double c = 0.5 * (l + h);
      const double r = fmax(__dadd_ru(h, -c), __dadd_ru(c, -l));
      const double ac = fabs(c), U = __dadd_ru(ac, r);
      if (f.kind == F_VAND) {
        double p = pow_rn(ac, e);
        if (c < 0 && (e & 1)) p = -p;
        v = tf32_rn((float)p);
      } else if (f.kind == F_DIFF) {
        const double pu = pow_dir(U, e, true), pc = pow_dir(ac, e, false);
        double d = __dadd_ru(pu, -pc);
        d = __dadd_ru(d, __dmul_ru((double)kKappa, pow_dir(ac, e, true)));
        if (f.extra > 0) d = __dadd_ru(d, __dmul_ru(f.extra, pu));
        v = tf32_ru_pos(__double2float_ru(d));
      } else {
        v = tf32_ru_pos(__double2float_ru(pow_dir(U, e, true)));
      }
    }
    const int k = f.koff + e;
    f.out[f.layout_b ? b_off(t, k, f.nk, f.NT) : a_off(t, k, f.nk)] = v;
  }
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sm_count() * 16) b = (int64_t)sm_count() * 16;
  if (b < 1) b = 1;
  return (int)b;
}

int launch_factors(const FactorArgs &f, cudaStream_t s) {
  k_factors<<<grid_for(f.rows * f.Kp), 256, 0, s>>>(f);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

template <int EPI>
int launch_mode(const TcArgs &a, cudaStream_t s) {
  const size_t need = (size_t)kStages * kG * (kAStep + a.NT * 32) + 64;
  // a 512-column TMEM allocation must not wait on a second resident block: ask for more than
  // half of the SM's shared memory then
  const size_t smem = a.NT > 128 ? std::max<size_t>(need, 120 * 1024) : need;
  const int64_t blocks = a.batches * a.mtiles * a.ntiles;
  if (blocks > 0x7fffffffll) {
    set_error("dense level: %lld tiles exceed one launch", (long long)blocks);
    return VX_EOVERFLOW;
  }
  k_tc_mode<EPI><<<(unsigned)blocks, 128, smem, s>>>(a);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

inline int roundup(int x, int m) { return (x + m - 1) / m * m; }

// The shared-memory limit of the four tensor-core kernels, set outside any stream capture.
int set_tc_attributes() {
  const int lim = 200 * 1024;
  VX_CUDA(cudaFuncSetAttribute(k_tc_mode<EPI_NEXT_B>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  VX_CUDA(cudaFuncSetAttribute(k_tc_mode<EPI_NEXT_A>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  VX_CUDA(cudaFuncSetAttribute(k_tc_mode<EPI_BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  VX_CUDA(cudaFuncSetAttribute(k_tc_mode<EPI_VALUES>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim));
  return VX_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// The plan: every operand buffer of the three modes for each polynomial, built once.
// ---------------------------------------------------------------------------------------
struct DensePolyOps {
  int D[3], Kp[3], nk[3];
  int N2p;                   // mode 2: NT (rows a3 of its B operand)
  int64_t ncols1, ntiles1;   // mode 1: columns (a2, a3) and their panels of 128
  float *B1 = nullptr, *B1a = nullptr;          // C^T and |C|^T (B layout, NT 128)
  float *V1 = nullptr, *F1 = nullptr;           // A layout
  float *V2 = nullptr, *F2 = nullptr;           // A layout, F2 = [D'|W]
  float *V3 = nullptr, *F3 = nullptr;           // B layout (NT 128), F3 = [D'|W]
};

struct DensePlan {
  int level = 0, npoly = 0;
  int64_t N = 0;
  double lo[3], w[3];
  std::vector<DensePolyOps> P;
  float *B2 = nullptr, *B2r = nullptr, *A3 = nullptr, *A3r = nullptr;  // intermediates
  std::vector<void *> mem;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  // the prefilter's launch sequence captured as a CUDA graph (for the mask it writes)
  cudaGraphExec_t graph = nullptr;
  uint32_t *graph_mask = nullptr;
};

static int plan_alloc(DensePlan *p, float **out, size_t floats, cudaStream_t s) {
  void *m = nullptr;
  VX_CHECK(dmalloc(&m, std::max<size_t>(floats, 1) * sizeof(float), s));
  p->mem.push_back(m);
  p->bytes += floats * sizeof(float);
  VX_CUDA(cudaMemsetAsync(m, 0, std::max<size_t>(floats, 1) * sizeof(float), s));
  *out = (float *)m;
  return VX_OK;
}

void dense_plan_free(DensePlan *p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (void *m : p->mem) dfree(m, p->stream);
  delete p;
}

int dense_plan_create(int npoly, const DenseHostPoly *polys, int level, const double *domain,
                      cudaStream_t s, DensePlan **out) {
  *out = nullptr;
  if (level < 5 || level > 12) {
    set_error("dense level: level %d outside [5, 12]", level);
    return VX_EINVAL;
  }
  DensePlan *p = new (std::nothrow) DensePlan();
  if (!p) {
    set_error("out of host memory");
    return VX_ENOMEM;
  }
  p->stream = s;
  if (set_tc_attributes() != VX_OK) {
    delete p;
    return VX_ECUDA;
  }
  p->level = level;
  p->npoly = npoly;
  p->N = (int64_t)1 << level;
  for (int i = 0; i < 3; ++i) {
    p->lo[i] = domain[2 * i];
    p->w[i] = (domain[2 * i + 1] - domain[2 * i]) / (double)p->N;
  }
  const int64_t N = p->N;
  const int64_t mtN = (N + 127) / 128;  // panels of 128 boxes along an axis
  int rc = VX_OK;
  size_t maxB2 = 0, maxB2r = 0, maxA3 = 0, maxA3r = 0;
  p->P.resize(npoly);
  for (int f = 0; f < npoly && rc == VX_OK; ++f) {
    DensePolyOps &o = p->P[f];
    const DenseHostPoly &hp = polys[f];
    for (int i = 0; i < 3; ++i) {
      o.D[i] = 0;
      for (int64_t t = 0; t < hp.nterms; ++t) o.D[i] = std::max(o.D[i], (int)hp.exps[t * 3 + i]);
      o.Kp[i] = roundup(o.D[i] + 1, 8);
      o.nk[i] = o.Kp[i] / 8;
    }
    if (o.D[2] + 1 > 256) {
      set_error("dense level: degree %d in x3 exceeds 255", o.D[2]);
      rc = VX_EINVAL;
      break;
    }
    o.N2p = roundup(o.D[2] + 1, 16);
    o.ncols1 = (int64_t)(o.D[1] + 1) * (o.D[2] + 1);
    o.ntiles1 = (o.ncols1 + 127) / 128;
    // mode 1 B operands from the coefficients, rounded to TF32 (the rounding, below 2^-10.9
    // of each coefficient, is charged to mode 1's radius factor)
    const size_t b1 = (size_t)o.ntiles1 * o.nk[0] * 128 * 8;
    std::vector<float> hb(b1, 0.f), hba(b1, 0.f);
    for (int64_t t = 0; t < hp.nterms; ++t) {
      const int a1 = hp.exps[t * 3], a2 = hp.exps[t * 3 + 1], a3 = hp.exps[t * 3 + 2];
      const int64_t j = (int64_t)a2 * (o.D[2] + 1) + a3;
      const int64_t off = b_off(j, a1, o.nk[0], 128);
      const float v = tf32_rn((float)hp.coefs[t]);
      hb[off] += v;  // repeated monomials are summed (in binary32, then again rounded)
      hba[off] = fabsf(tf32_rn(hb[off]));
      hb[off] = tf32_rn(hb[off]);
    }
    rc = plan_alloc(p, &o.B1, b1, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.B1a, b1, s);
    if (rc == VX_OK) {
      cudaError_t e = cudaMemcpyAsync(o.B1, hb.data(), b1 * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(o.B1a, hba.data(), b1 * 4, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors go out of scope
      if (e != cudaSuccess) {
        set_error("dense level: upload failed: %s", cudaGetErrorString(e));
        rc = VX_ECUDA;
      }
    }
    // factor matrices
    const size_t fa1 = (size_t)mtN * o.nk[0] * 1024, fa2 = (size_t)mtN * o.nk[1] * 1024;
    const size_t fb3 = (size_t)mtN * o.nk[2] * 1024;
    if (rc == VX_OK) rc = plan_alloc(p, &o.V1, fa1, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.F1, fa1, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.V2, fa2, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.F2, 2 * fa2, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.V3, fb3, s);
    if (rc == VX_OK) rc = plan_alloc(p, &o.F3, 2 * fb3, s);
    for (int ax = 0; ax < 3 && rc == VX_OK; ++ax) {
      FactorArgs fa{};
      fa.lo = p->lo[ax];
      fa.w = p->w[ax];
      fa.N = N;
      fa.rows = mtN * 128;
      fa.D = o.D[ax];
      fa.Kp = o.Kp[ax];
      fa.layout_b = ax == 2;
      fa.NT = 128;
      float *V = ax == 0 ? o.V1 : (ax == 1 ? o.V2 : o.V3);
      float *F = ax == 0 ? o.F1 : (ax == 1 ? o.F2 : o.F3);
      fa.kind = F_VAND;
      fa.out = V;
      fa.nk = o.nk[ax];
      fa.koff = 0;
      rc = launch_factors(fa, s);
      fa.kind = F_DIFF;
      fa.out = F;
      fa.nk = ax == 0 ? o.nk[0] : 2 * o.nk[ax];
      fa.extra = ax == 0 ? 0x1p-10 : 0.0;  // mode 1: the coefficients' TF32 rounding
      if (rc == VX_OK) rc = launch_factors(fa, s);
      if (ax > 0 && rc == VX_OK) {
        fa.kind = F_POW;
        fa.koff = o.Kp[ax];
        fa.extra = 0.0;
        rc = launch_factors(fa, s);
      }
    }
    maxB2 = std::max(maxB2, (size_t)N * o.nk[1] * o.N2p * 8);
    maxB2r = std::max(maxB2r, (size_t)N * 2 * o.nk[1] * o.N2p * 8);
    maxA3 = std::max(maxA3, (size_t)(N * N / 128) * o.nk[2] * 1024);
    maxA3r = std::max(maxA3r, (size_t)(N * N / 128) * 2 * o.nk[2] * 1024);
  }
  if (rc == VX_OK) rc = plan_alloc(p, &p->B2, maxB2, s);
  if (rc == VX_OK) rc = plan_alloc(p, &p->B2r, maxB2r, s);
  if (rc == VX_OK) rc = plan_alloc(p, &p->A3, maxA3, s);
  if (rc == VX_OK) rc = plan_alloc(p, &p->A3r, maxA3r, s);
  if (rc != VX_OK) {
    dense_plan_free(p);
    return rc;
  }
  *out = p;
  return VX_OK;
}

int64_t dense_plan_bytes(const DensePlan *p) { return (int64_t)p->bytes; }
int dense_plan_level(const DensePlan *p) { return p->level; }

// The three modes of polynomial f; mode 3 writes bits (mask) or values (v_mid, v_rad).
static int run_poly(const DensePlan *p, int f, uint32_t *mask, float *v_mid, float *v_rad,
                    cudaStream_t s) {
  const DensePolyOps &o = p->P[f];
  const int64_t N = p->N;
  const int64_t mtN = (N + 127) / 128;
  // the padding of the intermediates must read as zero for every polynomial
  const size_t b2 = (size_t)N * o.nk[1] * o.N2p * 8;
  if (f > 0) {
    VX_CUDA(cudaMemsetAsync(p->B2, 0, b2 * 4, s));
    VX_CUDA(cudaMemsetAsync(p->B2r, 0, 2 * b2 * 4, s));
  }
  // mode 1: t1 x (a2, a3), inner a1
  TcArgs a{};
  a.A = {o.V1, (int64_t)o.nk[0] * 1024, 0};
  a.Ar = {o.F1, (int64_t)o.nk[0] * 1024, 0};
  a.B = {o.B1, (int64_t)o.nk[0] * 128 * 8, 0};
  a.Br = {o.B1a, (int64_t)o.nk[0] * 128 * 8, 0};
  a.nk = o.nk[0];
  a.nkr = o.nk[0];
  a.NT = 128;
  a.mtiles = (int)mtN;
  a.ntiles = (int)o.ntiles1;
  a.batches = 1;
  a.idesc = idesc_tf32(128, 128);
  a.N = N;
  a.D3p1 = o.D[2] + 1;
  a.ncols = o.ncols1;
  a.nk_next = o.nk[1];
  a.Kp_next = o.Kp[1];
  a.NT_next = o.N2p;
  a.o_mid = p->B2;
  a.o_rad = p->B2r;
  a.o_mid_bstride = (int64_t)o.nk[1] * o.N2p * 8;
  a.o_rad_bstride = 2 * a.o_mid_bstride;
  VX_CHECK(launch_mode<EPI_NEXT_B>(a, s));
  // mode 2: per t1, t2 x a3, inner a2
  TcArgs b{};
  b.A = {o.V2, (int64_t)o.nk[1] * 1024, 0};
  b.Ar = {o.F2, (int64_t)2 * o.nk[1] * 1024, 0};
  b.B = {p->B2, 0, (int64_t)o.nk[1] * o.N2p * 8};
  b.Br = {p->B2r, 0, (int64_t)2 * o.nk[1] * o.N2p * 8};
  b.nk = o.nk[1];
  b.nkr = 2 * o.nk[1];
  b.NT = o.N2p;
  b.mtiles = (int)mtN;
  b.ntiles = 1;
  b.batches = N;
  b.idesc = idesc_tf32(128, (uint32_t)o.N2p);
  b.N = N;
  b.nk_next = o.nk[2];
  b.Kp_next = o.Kp[2];
  b.o_mid = p->A3;
  b.o_rad = p->A3r;
  VX_CHECK(launch_mode<EPI_NEXT_A>(b, s));
  // mode 3: (t1, t2) x t3, inner a3
  TcArgs c{};
  c.A = {p->A3, (int64_t)o.nk[2] * 1024, 0};
  c.Ar = {p->A3r, (int64_t)2 * o.nk[2] * 1024, 0};
  c.B = {o.V3, (int64_t)o.nk[2] * 128 * 8, 0};
  c.Br = {o.F3, (int64_t)2 * o.nk[2] * 128 * 8, 0};
  c.nk = o.nk[2];
  c.nkr = 2 * o.nk[2];
  c.NT = 128;
  c.mtiles = (int)(N * N / 128);
  c.ntiles = (int)mtN;
  c.batches = 1;
  c.idesc = idesc_tf32(128, 128);
  c.N = N;
  c.mask = mask;
  c.first = f == 0;
  c.v_mid = v_mid;
  c.v_rad = v_rad;
  if (mask) return launch_mode<EPI_BITS>(c, s);
  return launch_mode<EPI_VALUES>(c, s);
}

// The prefilter's launches (3 per polynomial, plus clears of the intermediates) are the same
// on every call for a given mask, so they are captured once as a CUDA graph and replayed.
int dense_prefilter(DensePlan *p, uint32_t *d_mask, cudaStream_t s) {
  if (!p->graph || p->graph_mask != d_mask) {
    if (p->graph) {
      cudaGraphExecDestroy(p->graph);
      p->graph = nullptr;
    }
    cudaStream_t cs = nullptr;
    VX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    int rc = VX_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = VX_ECUDA;
    for (int f = 0; f < p->npoly && rc == VX_OK; ++f) rc = run_poly(p, f, d_mask, nullptr, nullptr, cs);
    const cudaError_t e1 = cudaStreamEndCapture(cs, &g);
    if (rc == VX_OK && e1 != cudaSuccess) rc = VX_ECUDA;
    if (rc == VX_OK && cudaGraphInstantiate(&p->graph, g, 0) != cudaSuccess) {
      p->graph = nullptr;
      rc = VX_ECUDA;
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc != VX_OK) {
      if (rc == VX_ECUDA) set_error("dense prefilter: capturing the launch graph failed");
      return rc;
    }
    p->graph_mask = d_mask;
  }
  VX_CUDA(cudaGraphLaunch(p->graph, s));
  note_launch(3 * p->npoly);
  return VX_OK;
}

int dense_values(const DensePlan *p, int f, float *d_mid, float *d_rad, cudaStream_t s) {
  if (f < 0 || f >= p->npoly) {
    set_error("dense values: polynomial %d outside [0, %d)", f, p->npoly);
    return VX_EINVAL;
  }
  return run_poly(p, f, nullptr, d_mid, d_rad, s);
}

int set_dense_wait_polls(int64_t polls) {
  const uint32_t v =
      polls < 0 ? kDenseWaitPolls : (polls > 0xffffffffll ? 0xffffffffu : (uint32_t)polls);
  VX_CUDA(cudaMemcpyToSymbol(g_vx_dense_wait_polls, &v, sizeof(v)));
  return VX_OK;
}

int take_dense_status(cudaStream_t s, int *status) {
  int v = 0;
  VX_CUDA(cudaMemcpyFromSymbolAsync(&v, g_vx_dense_status, sizeof(int), 0,
                                    cudaMemcpyDeviceToHost, s));
  VX_CUDA(cudaStreamSynchronize(s));
  if (v) {
    const int zero = 0;
    VX_CUDA(cudaMemcpyToSymbolAsync(g_vx_dense_status, &zero, sizeof(int), 0,
                                    cudaMemcpyHostToDevice, s));
    VX_CUDA(cudaStreamSynchronize(s));
  }
  *status = v;
  return VX_OK;
}

// ---------------------------------------------------------------------------------------
// Survivors of a bit mask as lexicographic box indices (t1, t2, t3): bit i of the mask is box
// i = (t1 N + t2) N + t3.  Blocks of 256 threads take 8 words per thread; a block's count,
// the scan of the block counts, then each thread writes its words' boxes in order.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int kMW = 8;  // words per thread
constexpr int kMB = 256;

__global__ void __launch_bounds__(kMB) k_mask_count(const uint32_t *__restrict__ mask,
                                                     int64_t nwords, int32_t *bsum) {
  __shared__ int32_t sw[kMB / 32];
  const int64_t w0 = ((int64_t)blockIdx.x * kMB + threadIdx.x) * kMW;
  int32_t c = 0;
#pragma unroll
  for (int j = 0; j < kMW; ++j)
    if (w0 + j < nwords) c += __popc(mask[w0 + j]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int i = 0; i < kMB / 32; ++i) t += sw[i];
    bsum[blockIdx.x] = t;
  }
}

// exclusive scan of the block counts in place (one block); total at bsum[nb]
__global__ void __launch_bounds__(1024) k_mask_scan(int32_t *bsum, int64_t nb) {
  __shared__ int32_t sw[32];
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = (int64_t)threadIdx.x * per, b1 = std::min<int64_t>(b0 + per, nb);
  int32_t sum = 0;
  for (int64_t i = b0; i < b1; ++i) sum += bsum[i];
  int32_t incl = sum;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sw[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t v = sw[lane], x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    sw[lane] = x - v;
  }
  __syncthreads();
  int32_t run = incl - sum + sw[warp];
  for (int64_t i = b0; i < b1; ++i) {
    const int32_t v = bsum[i];
    bsum[i] = run;
    run += v;
  }
  if (threadIdx.x == blockDim.x - 1) bsum[nb] = run;
}

__global__ void __launch_bounds__(kMB) k_mask_emit(const uint32_t *__restrict__ mask,
                                                    int64_t nwords, const int32_t *bsum,
                                                    int level, int32_t *tuples) {
  __shared__ int32_t sw[kMB / 32];
  const int64_t w0 = ((int64_t)blockIdx.x * kMB + threadIdx.x) * kMW;
  uint32_t m[kMW];
  int32_t c = 0;
#pragma unroll
  for (int j = 0; j < kMW; ++j) {
    m[j] = w0 + j < nwords ? mask[w0 + j] : 0u;
    c += __popc(m[j]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sw[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t t = 0;
    for (int i = 0; i < kMB / 32; ++i) {
      const int32_t v = sw[i];
      sw[i] = t;
      t += v;
    }
  }
  __syncthreads();
  int32_t pos = bsum[blockIdx.x] + sw[warp] + incl - c;
  const int64_t side = (int64_t)1 << level, mlo = side - 1;
#pragma unroll
  for (int j = 0; j < kMW; ++j) {
    uint32_t bits = m[j];
    while (bits) {
      const int q = __ffs(bits) - 1;
      bits &= bits - 1;
      const int64_t i = (w0 + j) * 32 + q;
      tuples[3 * (int64_t)pos] = (int32_t)(i >> (2 * level));
      tuples[3 * (int64_t)pos + 1] = (int32_t)((i >> level) & mlo);
      tuples[3 * (int64_t)pos + 2] = (int32_t)(i & mlo);
      ++pos;
    }
  }
}

__global__ void k_scatter_keep(const int32_t *__restrict__ tuples, int64_t n, int level,
                               const uint8_t *__restrict__ keep, uint8_t *__restrict__ out) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = (((int64_t)tuples[3 * j] << level) + tuples[3 * j + 1]) << level;
    out[i + tuples[3 * j + 2]] = keep[j];
  }
}
}  // namespace

int mask_tuples(const uint32_t *d_mask, int level, cudaStream_t s, int32_t **d_tuples,
                int64_t *n) {
  *d_tuples = nullptr;
  *n = 0;
  const int64_t nwords = ((int64_t)1 << (3 * level)) / 32;
  const int64_t nb = (nwords + (int64_t)kMB * kMW - 1) / ((int64_t)kMB * kMW);
  int32_t *bsum = nullptr;
  VX_CHECK(dmalloc((void **)&bsum, (size_t)(nb + 1) * sizeof(int32_t), s));
  k_mask_count<<<(unsigned)nb, kMB, 0, s>>>(d_mask, nwords, bsum);
  note_launch();
  k_mask_scan<<<1, 1024, 0, s>>>(bsum, nb);
  note_launch();
  int32_t total = 0;
  cudaError_t e = cudaMemcpyAsync(&total, bsum + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dfree(bsum, s);
    set_error("dense level: survivor count failed: %s", cudaGetErrorString(e));
    return VX_ECUDA;
  }
  int rc = VX_OK;
  if (total > 0) rc = dmalloc((void **)d_tuples, (size_t)total * 3 * sizeof(int32_t), s);
  if (rc == VX_OK && total > 0) {
    k_mask_emit<<<(unsigned)nb, kMB, 0, s>>>(d_mask, nwords, bsum, level, *d_tuples);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("dense level: survivor emit launch failed");
      rc = VX_ECUDA;
    }
  }
  dfree(bsum, s);
  if (rc == VX_OK) *n = total;
  return rc;
}

int scatter_keep_grid(const int32_t *d_tuples, int64_t n, int level, const uint8_t *d_keep,
                      uint8_t *d_out, cudaStream_t s) {
  if (n == 0) return VX_OK;
  k_scatter_keep<<<grid_for(n), 256, 0, s>>>(d_tuples, n, level, d_keep, d_out);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

}  // namespace vx
