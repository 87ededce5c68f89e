// vx_csf.cu -- the integer side of one subdivision level: CSF construction from sorted box
// indices (Sec. 2.1), and Algorithm 3's step from the boxes that pass C0 to the next level's
// tree, without sorting.
//
// Both are scans over 0/1 flags: a reduce-then-scan over tiles of 2048 entries (256 threads
// x 8 entries), up to 4 flag channels at once (one per CSF depth), warp-shuffle scans inside
// a block and one small kernel scanning the tile sums.
//
// Bisection (Algorithm 3, "set of boxes bisected from the boxes in S"): a kept depth-d node
// with label i becomes the two nodes 2i and 2i+1, each carrying a copy of its kept subtree.
// In lexicographic order a new depth-t node (path p_0..p_t of kept nodes, bits b_0..b_t)
// sits at
//     sum_{a=0..t} [ 2^(t-a+1) (F_t(p_a) - F_t(p_{a-1})) + b_a 2^(t-a) D_t(p_a) ]
// where F_t(p) is the rank of p's first kept depth-t descendant (F_t(root) = 0) and D_t(p)
// the number of them: the nodes before it are the copies of the subtrees of earlier siblings
// of each ancestor (2^(t-a+1) copies per kept depth-t descendant) and, inside an ancestor's
// pair, the copies under the lower bit.  Ranks and first descendants come from one scan of
// the keep flags, so every new node is written straight to its place.
#include <cuda_runtime.h>

#include "vx_internal.cuh"

namespace vx {
namespace {

constexpr int ST = 256;
constexpr int SI = 8;
constexpr int STILE = ST * SI;

__device__ __forceinline__ int32_t warp_incl_scan(int32_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t u = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += u;
  }
  return v;
}

__device__ __forceinline__ int32_t warp_sum(int32_t v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <int C, class Src>
__global__ void __launch_bounds__(ST) k_scan_reduce(Src src, int64_t n, int32_t *tsum,
                                                    int64_t ntiles) {
  __shared__ int32_t sw[C][ST / 32];
  const int64_t tile = blockIdx.x;
  const int64_t i0 = tile * STILE + (int64_t)threadIdx.x * SI;
  int32_t cnt[C];
#pragma unroll
  for (int c = 0; c < C; ++c) cnt[c] = 0;
  for (int j = 0; j < SI; ++j) {
    const int64_t i = i0 + j;
    if (i < n) {
      const unsigned m = src.flags(i, true);
#pragma unroll
      for (int c = 0; c < C; ++c) cnt[c] += (m >> c) & 1u;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    int32_t v = warp_sum(cnt[c]);
    if (lane == 0) sw[c][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      int32_t v = lane < ST / 32 ? sw[c][lane] : 0;
      v = warp_sum(v);
      if (lane == 0) tsum[c * ntiles + tile] = v;
    }
  }
}

// In-place exclusive scan of each channel's tile sums; totals[c] = channel total.
template <int C>
__global__ void __launch_bounds__(1024) k_scan_tiles(int32_t *tsum, int64_t ntiles,
                                                     int32_t *totals) {
  __shared__ int32_t sw[32];
  __shared__ int32_t s_total;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < C; ++c) {
    int32_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += 1024) {
      const int64_t i = b + threadIdx.x;
      const int32_t v = i < ntiles ? tsum[c * ntiles + i] : 0;
      int32_t incl = warp_incl_scan(v);
      if (lane == 31) sw[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        int32_t w = sw[lane];
        int32_t wi = warp_incl_scan(w);
        sw[lane] = wi - w;
        if (lane == 31) s_total = wi;
      }
      __syncthreads();
      incl += sw[warp];
      if (i < ntiles) tsum[c * ntiles + i] = carry + incl - v;
      carry += s_total;
      __syncthreads();
    }
    if (threadIdx.x == 0) totals[c] = carry;
  }
}

template <int C, class Src, class Emit>
__global__ void __launch_bounds__(ST) k_scan_emit(Src src, Emit em, int64_t n,
                                                  const int32_t *toff, int64_t ntiles) {
  __shared__ int32_t sw[C][ST / 32];
  const int64_t tile = blockIdx.x;
  const int64_t i0 = tile * STILE + (int64_t)threadIdx.x * SI;
  unsigned m[SI];
  int32_t cnt[C];
#pragma unroll
  for (int c = 0; c < C; ++c) cnt[c] = 0;
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    const int64_t i = i0 + j;
    m[j] = i < n ? src.flags(i, false) : 0u;
#pragma unroll
    for (int c = 0; c < C; ++c) cnt[c] += (m[j] >> c) & 1u;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t pre[C];
#pragma unroll
  for (int c = 0; c < C; ++c) {
    int32_t incl = warp_incl_scan(cnt[c]);
    pre[c] = incl - cnt[c];
    if (lane == 31) sw[c][warp] = incl;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      int32_t v = lane < ST / 32 ? sw[c][lane] : 0;
      int32_t s = warp_incl_scan(v);
      if (lane < ST / 32) sw[c][lane] = s - v;
    }
  }
  __syncthreads();
  int32_t run[C];
#pragma unroll
  for (int c = 0; c < C; ++c) run[c] = toff[c * ntiles + tile] + sw[c][warp] + pre[c];
#pragma unroll
  for (int j = 0; j < SI; ++j) {
    const int64_t i = i0 + j;
    if (i < n) {
      em(i, m[j], run);
#pragma unroll
      for (int c = 0; c < C; ++c) run[c] += (m[j] >> c) & 1u;
    }
  }
}

// Pinned staging for the few counts the host needs (one buffer per host thread).
int32_t *pinned_counts() {
  static thread_local int32_t *p = nullptr;
  if (!p) {
    if (cudaHostAlloc((void **)&p, 64 * sizeof(int32_t), cudaHostAllocDefault) != cudaSuccess) {
      p = nullptr;
    }
  }
  return p;
}

// Runs reduce + tile scan; leaves the tile offsets in *d_scratch (caller frees) and copies the
// channel totals to h_totals (synchronising the stream).
template <int C, class Src>
int scan_prepare(const Src &src, int64_t n, cudaStream_t s, int32_t **d_scratch,
                 int64_t *ntiles_out, int32_t *h_totals, const int32_t *d_extra = nullptr,
                 int32_t *h_extra = nullptr) {
  const int64_t ntiles = (n + STILE - 1) / STILE;
  *ntiles_out = ntiles;
  *d_scratch = nullptr;
  int32_t *pin = pinned_counts();
  if (!pin) {
    set_error("cudaHostAlloc of the count staging buffer failed");
    return VX_ENOMEM;
  }
  if (ntiles == 0) {
    for (int c = 0; c < C; ++c) h_totals[c] = 0;
    if (h_extra) *h_extra = 0;
    return VX_OK;
  }
  if (ntiles > INT32_MAX) {
    set_error("scan of %lld entries is too large", (long long)n);
    return VX_EOVERFLOW;
  }
  int32_t *buf = nullptr;
  VX_CHECK(dmalloc((void **)&buf, (size_t)(C * ntiles + C) * sizeof(int32_t), s));
  *d_scratch = buf;
  k_scan_reduce<C, Src><<<(unsigned)ntiles, ST, 0, s>>>(src, n, buf, ntiles);
  note_launch();
  VX_LAUNCH_CHECK();
  k_scan_tiles<C><<<1, 1024, 0, s>>>(buf, ntiles, buf + C * ntiles);
  note_launch();
  VX_LAUNCH_CHECK();
  VX_CUDA(cudaMemcpyAsync(pin, buf + C * ntiles, C * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  if (d_extra)
    VX_CUDA(cudaMemcpyAsync(pin + C, d_extra, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  VX_CUDA(cudaStreamSynchronize(s));
  for (int c = 0; c < C; ++c) h_totals[c] = pin[c];
  if (h_extra) *h_extra = d_extra ? pin[C] : 0;
  return VX_OK;
}

template <int C, class Src, class Emit>
int scan_emit(const Src &src, const Emit &em, int64_t n, const int32_t *d_scratch,
              int64_t ntiles, cudaStream_t s) {
  if (ntiles == 0) return VX_OK;
  k_scan_emit<C, Src, Emit><<<(unsigned)ntiles, ST, 0, s>>>(src, em, n, d_scratch, ntiles);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

// ---------------------------------------------------------------------------------------
// csf_build: channel d flags the tuples that start a depth-d node (their first d+1
// coordinates differ from the previous tuple's).
// ---------------------------------------------------------------------------------------
struct BuildSrc {
  const int32_t *t;
  int32_t k, side;
  int32_t *err;
  __device__ unsigned flags(int64_t i, bool check) const {
    const unsigned all = (1u << k) - 1u;
    if (check) {
      for (int c = 0; c < k; ++c) {
        int32_t v = t[i * k + c];
        if (v < 0 || v >= side) atomicOr(err, 1);
      }
    }
    if (i == 0) return all;
    int fd = k;
    for (int c = 0; c < k; ++c) {
      if (t[i * k + c] != t[(i - 1) * k + c]) {
        fd = c;
        break;
      }
    }
    if (check && (fd == k || t[i * k + fd] < t[(i - 1) * k + fd])) atomicOr(err, 2);
    if (fd == k) return 0u;
    return all & ~((1u << fd) - 1u);
  }
};

struct BuildEmit {
  CsfView out;
  const int32_t *t;
  __device__ void operator()(int64_t i, unsigned m, const int32_t *excl) const {
    const int k = out.k;
    for (int d = 0; d < k; ++d) {
      if (!((m >> d) & 1u)) continue;
      const int32_t node = excl[d];
      out.lab[d][node] = t[i * k + d];
      if (d > 0) {
        const int32_t pnode = excl[d - 1] + (int32_t)((m >> (d - 1)) & 1u) - 1;
        out.par[d][node] = pnode;
        if ((m >> (d - 1)) & 1u) out.ptr[d - 1][pnode] = node;  // first child of a new parent
      }
    }
  }
};

struct Sentinels {
  int32_t *p[VX_KMAX];
  int64_t at[VX_KMAX];
  int32_t val[VX_KMAX];
};

__global__ void k_set_sentinels(Sentinels s, int n) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    for (int i = 0; i < n; ++i) s.p[i][s.at[i]] = s.val[i];
}

}  // namespace

int set_ptr_sentinels(const CsfView &v, cudaStream_t s) {
  Sentinels S;
  int n = 0;
  for (int d = 0; d + 1 < v.k; ++d) {
    S.p[n] = v.ptr[d];
    S.at[n] = v.N[d];
    S.val[n] = (int32_t)v.N[d + 1];
    ++n;
  }
  if (n == 0) return VX_OK;
  k_set_sentinels<<<1, 32, 0, s>>>(S, n);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

namespace {

template <int C>
int build_c(int k, int level, const int32_t *d_tuples, int64_t n, cudaStream_t s, CsfObj *out,
            Timer *tm) {
  int32_t *d_err = nullptr;
  VX_CHECK(dmalloc((void **)&d_err, sizeof(int32_t), s));
  VX_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int32_t), s));
  BuildSrc src{d_tuples, (int32_t)k, (int32_t)(1 << level), d_err};
  int32_t *scratch = nullptr;
  int64_t ntiles = 0;
  int32_t tot[C];
  if (tm && tm->on) VX_CHECK(tm->begin(KK_CSF_BUILD, n * k * 4));
  int32_t herr = 0;
  int rc = scan_prepare<C>(src, n, s, &scratch, &ntiles, tot, d_err, &herr);
  if (rc == VX_OK && herr) {
    set_error(herr & 1 ? "csf_build: a tuple coordinate is outside [0, 2^level)"
                       : "csf_build: tuples are not strictly increasing in lexicographic order");
    rc = VX_EINVAL;
  }
  if (rc == VX_OK) {
    int64_t N[VX_KMAX] = {0};
    for (int d = 0; d < k; ++d) N[d] = tot[d];
    rc = csf_alloc(out, k, level, N, s);
  }
  if (rc == VX_OK) rc = scan_emit<C>(src, BuildEmit{out->v, d_tuples}, n, scratch, ntiles, s);
  if (rc == VX_OK) rc = set_ptr_sentinels(out->v, s);
  if (rc == VX_OK && tm && tm->on) rc = tm->end();
  dfree(scratch, s);
  dfree(d_err, s);
  return rc;
}

// ---------------------------------------------------------------------------------------
// Prune: node flags of every depth in one array (depth d at offset off[d]); channel d
// counts the kept nodes of depth d, so the exclusive scan is each node's rank g_d.
// ---------------------------------------------------------------------------------------
struct Segs {
  int64_t off[VX_KMAX + 1];
  int32_t k;
};

struct FlagSrc {
  const uint8_t *f;
  Segs sg;
  __device__ int depth_of(int64_t i) const {
    int d = 0;
    while (d + 1 < sg.k && i >= sg.off[d + 1]) ++d;
    return d;
  }
  __device__ unsigned flags(int64_t i, bool) const {
    return f[i] ? (1u << depth_of(i)) : 0u;
  }
};

struct RankEmit {
  int32_t *rank;
  FlagSrc src;
  __device__ void operator()(int64_t i, unsigned m, const int32_t *excl) const {
    rank[i] = excl[src.depth_of(i)];
  }
};

// keep flags upward: a node is kept iff some leaf below it is kept
__global__ void k_mark_up(CsfView c, const uint8_t *__restrict__ keep, uint8_t *flags, Segs sg) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint8_t kp = keep[i] ? 1 : 0;
    flags[sg.off[k - 1] + i] = kp;
    if (!kp) continue;
    int64_t p = i;
    for (int d = k - 1; d > 0; --d) {
      p = c.par[d][p];
      uint8_t *f = flags + sg.off[d - 1] + p;
      if (*(volatile uint8_t *)f) break;  // whoever set it carries on upward
      *f = 1;
    }
  }
}

// kptr[d][g_d(p)] = rank of the first kept child of kept node p (depth d < k-1)
__global__ void k_kptr(CsfView c, const uint8_t *__restrict__ flags, const int32_t *__restrict__ rank,
                       Segs sg, int d, int32_t *kptr) {
  const int64_t n = c.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    if (!flags[sg.off[d] + p]) continue;
    kptr[rank[sg.off[d] + p]] = rank[sg.off[d + 1] + c.ptr[d][p]];
  }
}

struct KptrSet {
  const int32_t *k[VX_KMAX];  // kptr[d], n_d + 1 entries (last = n_{d+1})
};

__device__ __forceinline__ int32_t chain(const KptrSet &K, int a, int t, int32_t r) {
  for (int e = a; e < t; ++e) r = K.k[e][r];
  return r;
}

// Bisection of depth d: every kept depth-d node writes its 2^(d+1) copies.
__global__ void k_split(CsfView in, const uint8_t *__restrict__ flags,
                        const int32_t *__restrict__ rank, Segs sg, KptrSet K, int d, CsfView out) {
  const int k = in.k;
  const int64_t n = in.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    if (!flags[sg.off[d] + p]) continue;
    int64_t path[VX_KMAX];
    int32_t g[VX_KMAX];
    path[d] = p;
    for (int a = d; a > 0; --a) path[a - 1] = in.par[a][path[a]];
    for (int a = 0; a <= d; ++a) g[a] = rank[sg.off[a] + path[a]];
    // F_t(p_a) and D_t(p_a) for t = d-1, d, d+1
    int64_t base_d = 0, base_m = 0, base_p = 0;
    int64_t Dd[VX_KMAX], Dm[VX_KMAX], Dp[VX_KMAX];
    int64_t prevF_d = 0, prevF_m = 0, prevF_p = 0;
    for (int a = 0; a <= d; ++a) {
      const int64_t Fd = chain(K, a, d, g[a]);
      Dd[a] = chain(K, a, d, g[a] + 1) - Fd;
      base_d += (Fd - prevF_d) << (d - a + 1);
      prevF_d = Fd;
      if (a < d) {
        const int64_t Fm = chain(K, a, d - 1, g[a]);
        Dm[a] = chain(K, a, d - 1, g[a] + 1) - Fm;
        base_m += (Fm - prevF_m) << (d - a);
        prevF_m = Fm;
      }
      if (d + 1 < k) {
        const int64_t Fp = chain(K, a, d + 1, g[a]);
        Dp[a] = chain(K, a, d + 1, g[a] + 1) - Fp;
        base_p += (Fp - prevF_p) << (d - a + 2);
        prevF_p = Fp;
      }
    }
    const int32_t lab2 = 2 * in.lab[d][p];
    const int nb = 1 << (d + 1);
    for (int b = 0; b < nb; ++b) {
      int64_t idx = base_d, pidx = base_m, cidx = base_p;
      for (int a = 0; a <= d; ++a) {
        const int64_t bit = (b >> (d - a)) & 1;
        idx += bit * (Dd[a] << (d - a));
        if (a < d) pidx += bit * (Dm[a] << (d - 1 - a));
        if (d + 1 < k) cidx += bit * (Dp[a] << (d - a + 1));
      }
      out.lab[d][idx] = lab2 + (b & 1);
      if (d > 0) out.par[d][idx] = (int32_t)pidx;
      if (d + 1 < k) out.ptr[d][idx] = (int32_t)cidx;
    }
  }
}

// Compaction of depth d: kept node p goes to its rank.
__global__ void k_gather(CsfView in, const uint8_t *__restrict__ flags,
                         const int32_t *__restrict__ rank, Segs sg, int d, CsfView out,
                         int32_t *index) {
  const int64_t n = in.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
    if (!flags[sg.off[d] + p]) continue;
    const int32_t r = rank[sg.off[d] + p];
    out.lab[d][r] = in.lab[d][p];
    if (d > 0) out.par[d][r] = rank[sg.off[d - 1] + in.par[d][p]];
    if (index && d == in.k - 1) index[r] = (int32_t)p;
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <int C>
int prune_c(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
            cudaStream_t s, CsfObj *out, Timer *tm) {
  const int k = in.k;
  Segs sg;
  sg.k = k;
  sg.off[0] = 0;
  for (int d = 0; d < k; ++d) sg.off[d + 1] = sg.off[d] + in.N[d];
  for (int d = k + 1; d <= VX_KMAX; ++d) sg.off[d] = sg.off[k];
  const int64_t total = sg.off[k];
  if (total > INT32_MAX) {
    set_error("tree with %lld nodes exceeds 32-bit indices", (long long)total);
    return VX_EOVERFLOW;
  }
  if (in.N[k - 1] == 0) {  // empty level: empty result
    int64_t N[VX_KMAX] = {0};
    VX_CHECK(csf_alloc(out, k, in.level + (split ? 1 : 0), N, s));
    return set_ptr_sentinels(out->v, s);
  }
  uint8_t *flags = nullptr;
  int32_t *rank = nullptr, *kptr = nullptr, *scratch = nullptr;
  int rc = VX_OK;
  if (tm && tm->on) VX_CHECK(tm->begin(KK_PRUNE, total * 9));
  rc = dmalloc((void **)&flags, (size_t)total, s);
  if (rc == VX_OK) rc = dmalloc((void **)&rank, (size_t)total * sizeof(int32_t), s);
  if (rc == VX_OK && sg.off[k - 1] > 0) {
    cudaError_t e = cudaMemsetAsync(flags, 0, (size_t)sg.off[k - 1], s);
    if (e != cudaSuccess) {
      set_error("cudaMemsetAsync failed: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  if (rc == VX_OK) {
    k_mark_up<<<blocks_for(in.N[k - 1]), 256, 0, s>>>(in, d_keep, flags, sg);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("mark-up kernel launch failed");
      rc = VX_ECUDA;
    }
  }
  FlagSrc src{flags, sg};
  int64_t ntiles = 0;
  int32_t nk[C];
  if (rc == VX_OK) rc = scan_prepare<C>(src, total, s, &scratch, &ntiles, nk);
  if (rc == VX_OK) rc = scan_emit<C>(src, RankEmit{rank, src}, total, scratch, ntiles, s);
  // kept-tree first-child pointers
  KptrSet K{};
  int64_t koff[VX_KMAX + 1] = {0};
  for (int d = 0; d + 1 < k; ++d) koff[d + 1] = koff[d] + nk[d] + 1;
  int64_t newN[VX_KMAX] = {0};
  if (rc == VX_OK) {
    for (int d = 0; d < k; ++d) {
      newN[d] = split ? ((int64_t)nk[d] << (d + 1)) : nk[d];
      if (newN[d] > INT32_MAX) {
        set_error("next level would have %lld nodes at depth %d (32-bit indices)",
                  (long long)newN[d], d + 1);
        rc = VX_EOVERFLOW;
      }
    }
  }
  if (rc == VX_OK && tm && tm->on) rc = tm->end();
  if (rc == VX_OK) rc = csf_alloc(out, k, in.level + (split ? 1 : 0), newN, s);
  if (rc == VX_OK && k > 1) {
    if (split) {
      rc = dmalloc((void **)&kptr, (size_t)(koff[k - 1] > 0 ? koff[k - 1] : 1) * sizeof(int32_t), s);
      for (int d = 0; d + 1 < k && rc == VX_OK; ++d) K.k[d] = kptr + koff[d];
    } else {
      for (int d = 0; d + 1 < k; ++d) K.k[d] = out->v.ptr[d];
    }
  }
  if (rc == VX_OK && tm && tm->on) rc = tm->begin(split ? KK_SPLIT : KK_COMPACT,
                                                  split ? (newN[k - 1] * 8 + total * 9) : total * 13);
  for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
    k_kptr<<<blocks_for(in.N[d]), 256, 0, s>>>(in, flags, rank, sg, d, (int32_t *)K.k[d]);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("kptr kernel launch failed");
      rc = VX_ECUDA;
    }
    if (rc == VX_OK) {
      Sentinels S;
      S.p[0] = (int32_t *)K.k[d];
      S.at[0] = nk[d];
      S.val[0] = nk[d + 1];
      k_set_sentinels<<<1, 32, 0, s>>>(S, 1);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) rc = VX_ECUDA;
    }
  }
  for (int d = 0; d < k && rc == VX_OK; ++d) {
    if (split)
      k_split<<<blocks_for(in.N[d]), 256, 0, s>>>(in, flags, rank, sg, K, d, out->v);
    else
      k_gather<<<blocks_for(in.N[d]), 256, 0, s>>>(in, flags, rank, sg, d, out->v, d_index);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("split/gather kernel launch failed: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  if (rc == VX_OK && split) rc = set_ptr_sentinels(out->v, s);
  if (rc == VX_OK && tm && tm->on) rc = tm->end();
  dfree(kptr, s);
  dfree(scratch, s);
  dfree(rank, s);
  dfree(flags, s);
  return rc;
}

__global__ void k_tuples(CsfView c, int32_t *t) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t p = i;
    for (int d = k - 1; d >= 0; --d) {
      t[i * k + d] = c.lab[d][p];
      if (d > 0) p = c.par[d][p];
    }
  }
}

// indices of the nonzero bytes, in increasing order
struct ByteFlagSrc {
  const uint8_t *f;
  __device__ unsigned flags(int64_t i, bool) const { return f[i] ? 1u : 0u; }
};
struct IndexEmit {
  int32_t *idx;
  __device__ void operator()(int64_t i, unsigned m, const int32_t *excl) const {
    if (m) idx[excl[0]] = (int32_t)i;
  }
};

__global__ void k_tuples_of(CsfView c, const int32_t *__restrict__ idx, int64_t n, int32_t *t) {
  const int k = c.k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t p = idx[i];
    for (int d = k - 1; d >= 0; --d) {
      t[i * k + d] = c.lab[d][p];
      if (d > 0) p = c.par[d][p];
    }
  }
}

// The complete tree of a level: depth d holds side^(d+1) nodes, node i has label i % side,
// parent i / side and children i*side .. i*side + side - 1.
__global__ void k_full_grid(CsfView c, int32_t side) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int d = 0; d < c.k; ++d) {
    const int64_t n = c.N[d];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
      if (i < n) {
        c.lab[d][i] = (int32_t)(i % side);
        if (d > 0) c.par[d][i] = (int32_t)(i / side);
      }
      if (d + 1 < c.k) c.ptr[d][i] = (int32_t)(i * side);
    }
  }
}

__global__ void k_scatter(const int32_t *__restrict__ index, const uint8_t *__restrict__ sub,
                          int64_t n, uint8_t *keep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    keep[index[i]] = sub[i];
}

}  // namespace

int csf_alloc(CsfObj *o, int k, int level, const int64_t *N, cudaStream_t s) {
  o->v = CsfView{};
  o->v.k = k;
  o->v.level = level;
  o->mem = nullptr;
  o->stream = s;
  size_t bytes = 0;
  auto round = [](size_t x) { return (x + 127) & ~(size_t)127; };
  for (int d = 0; d < k; ++d) {
    o->v.N[d] = N[d];
    bytes += round((size_t)N[d] * 4);
    if (d > 0) bytes += round((size_t)N[d] * 4);
    if (d + 1 < k) bytes += round((size_t)(N[d] + 1) * 4);
  }
  VX_CHECK(dmalloc(&o->mem, bytes > 0 ? bytes : 128, s));
  o->bytes = bytes > 0 ? bytes : 128;
  char *p = (char *)o->mem;
  for (int d = 0; d < k; ++d) {
    o->v.lab[d] = (int32_t *)p;
    p += round((size_t)N[d] * 4);
    if (d > 0) {
      o->v.par[d] = (int32_t *)p;
      p += round((size_t)N[d] * 4);
    }
    if (d + 1 < k) {
      o->v.ptr[d] = (int32_t *)p;
      p += round((size_t)(N[d] + 1) * 4);
    }
  }
  return VX_OK;
}

void csf_release(CsfObj *o) {
  if (o->mem) dfree(o->mem, o->stream);
  o->mem = nullptr;
}

int csf_build_dev(int k, int level, const int32_t *d_tuples, int64_t n, cudaStream_t s,
                  CsfObj *out, Timer *tm) {
  if (n > INT32_MAX) {
    set_error("csf_build: %lld tuples exceed 32-bit indices", (long long)n);
    return VX_EOVERFLOW;
  }
  switch (k) {
    case 1: return build_c<1>(k, level, d_tuples, n, s, out, tm);
    case 2: return build_c<2>(k, level, d_tuples, n, s, out, tm);
    case 3: return build_c<3>(k, level, d_tuples, n, s, out, tm);
    default: return build_c<4>(k, level, d_tuples, n, s, out, tm);
  }
}

int csf_prune(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
              cudaStream_t s, CsfObj *out, Timer *tm) {
  switch (in.k) {
    case 1: return prune_c<1>(in, d_keep, split, d_index, s, out, tm);
    case 2: return prune_c<2>(in, d_keep, split, d_index, s, out, tm);
    case 3: return prune_c<3>(in, d_keep, split, d_index, s, out, tm);
    default: return prune_c<4>(in, d_keep, split, d_index, s, out, tm);
  }
}

int csf_tuples_dev(const CsfView &c, int32_t *d_tuples, cudaStream_t s) {
  if (c.N[c.k - 1] == 0) return VX_OK;
  k_tuples<<<blocks_for(c.N[c.k - 1]), 256, 0, s>>>(c, d_tuples);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

int csf_full_grid_dev(int k, int level, cudaStream_t s, CsfObj *out) {
  int64_t N[VX_KMAX] = {0};
  int64_t n = 1;
  for (int d = 0; d < k; ++d) {
    n <<= level;
    if (n > INT32_MAX) {
      set_error("the full level-%d grid in %d variables has more than 2^31 boxes", level, k);
      return VX_EOVERFLOW;
    }
    N[d] = n;
  }
  VX_CHECK(csf_alloc(out, k, level, N, s));
  k_full_grid<<<blocks_for(N[k - 1] + 1), 256, 0, s>>>(out->v, 1 << level);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

int flag_indices(const uint8_t *d_flags, int64_t n, cudaStream_t s, int32_t **d_idx,
                 int64_t *count) {
  *d_idx = nullptr;
  *count = 0;
  if (n > INT32_MAX) {
    set_error("flag_indices: %lld entries exceed 32-bit indices", (long long)n);
    return VX_EOVERFLOW;
  }
  ByteFlagSrc src{d_flags};
  int32_t *scratch = nullptr;
  int64_t ntiles = 0;
  int32_t tot[1] = {0};
  int rc = scan_prepare<1>(src, n, s, &scratch, &ntiles, tot);
  if (rc == VX_OK && tot[0] > 0) {
    rc = dmalloc((void **)d_idx, (size_t)tot[0] * 4, s);
    if (rc == VX_OK) rc = scan_emit<1>(src, IndexEmit{*d_idx}, n, scratch, ntiles, s);
  }
  dfree(scratch, s);
  if (rc == VX_OK) *count = tot[0];
  return rc;
}

int csf_tuples_of(const CsfView &c, const int32_t *d_idx, int64_t n, int32_t *d_tuples,
                  cudaStream_t s) {
  if (n == 0) return VX_OK;
  k_tuples_of<<<blocks_for(n), 256, 0, s>>>(c, d_idx, n, d_tuples);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

int scatter_keep(const int32_t *d_index, const uint8_t *d_sub_keep, int64_t n, uint8_t *d_keep,
                 cudaStream_t s) {
  if (n == 0) return VX_OK;
  k_scatter<<<blocks_for(n), 256, 0, s>>>(d_index, d_sub_keep, n, d_keep);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

}  // namespace vx
