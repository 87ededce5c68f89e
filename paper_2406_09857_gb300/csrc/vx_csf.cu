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
// the keep flags, so every new node is written straight to its place.  The scan stores a rank
// per inner node and one count per 8-entry word of the leaves' flags (RankView); the kernels
// that place nodes take 32 consecutive flags per warp, one rank per warp and a ballot.
#include <cuda_runtime.h>

#include <algorithm>

#include "vx_internal.cuh"

namespace vx {
namespace {

constexpr int ST = 256;
constexpr int SI = 8;
constexpr int STILE = ST * SI;  // entries of one pass of a CTA
constexpr int SR = 8;           // at most SR passes per CTA: a scan tile is passes * STILE entries

// Passes per scan tile: several for large scans (fewer, longer-lived CTAs and fewer tile sums),
// one while that would leave fewer than 2048 tiles to spread over the GPU.
__host__ __device__ __forceinline__ int scan_passes(int64_t n) {
  const int64_t t1 = (n + STILE - 1) / STILE;
  const int64_t p = t1 / 2048;
  return (int)(p < 1 ? 1 : (p > SR ? SR : p));
}

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

// The SI entries of a thread (i0 .. i0+SI-1): a source may load them at once (load_items);
// the default asks for them one by one.
template <class Src>
__device__ __forceinline__ void load_items(const Src &src, int64_t i0, int64_t n, bool check,
                                           unsigned (&m)[SI]) {
#pragma unroll
  for (int j = 0; j < SI; ++j) m[j] = i0 + j < n ? src.flags(i0 + j, check) : 0u;
}

// An emitter may store the SI entries at once (emit_items); the default calls it per entry
// with the running exclusive counts.
template <int C, class Emit>
__device__ __forceinline__ void emit_items(const Emit &em, int64_t i0, int64_t n,
                                           const unsigned (&m)[SI], int32_t (&run)[C]) {
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

// A thread's SI entries in a scan: loaded (load), counted per channel (count) and handed to
// the emitter with the running exclusive counts (emit).  A source may specialise it (FlagSrc:
// eight flag bytes of one depth counted and ranked a word at a time).
template <int C, class Src>
struct ItemOps {
  unsigned m[SI];
  __device__ __forceinline__ void load(const Src &src, int64_t i0, int64_t n, bool check) {
    load_items(src, i0, n, check, m);
  }
  __device__ __forceinline__ void count(int32_t (&cnt)[C]) const {
#pragma unroll
    for (int j = 0; j < SI; ++j)
#pragma unroll
      for (int c = 0; c < C; ++c) cnt[c] += (m[j] >> c) & 1u;
  }
  template <class Emit>
  __device__ __forceinline__ void emit(const Emit &em, int64_t i0, int64_t n,
                                       int32_t (&run)[C]) const {
    emit_items<C>(em, i0, n, m, run);
  }
};

// A tile whose entries the source can count in a form of its own (32 flag bytes per thread
// and step): adds them to cnt and returns true.  Entries t0..t1-1.
template <int C, class Src>
__device__ __forceinline__ bool reduce_tile(const Src &, int64_t, int64_t, int32_t (&)[C]) {
  return false;
}

// The nonzero bytes among entries e0 .. e0+31 (< t1) of a byte array: byte j of word q as bit
// 8 (j) + 7 of nz[q] (two 16-byte loads when all 32 lie before t1; f 16-byte aligned, e0 a
// multiple of 32).
__device__ __forceinline__ void nonzero32(const uint8_t *f, int64_t e0, int64_t t1,
                                          uint32_t (&nz)[8]) {
  if (e0 + 32 <= t1) {
    const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(f + e0));
    const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(f + e0 + 16));
    const uint32_t w[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) nz[q] = (((w[q] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w[q]) & 0x80808080u;
  } else {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      nz[q] = 0u;
      for (int j = 0; j < 4; ++j) {
        const int64_t i = e0 + 4 * q + j;
        if (i < t1 && f[i]) nz[q] |= 0x80u << (8 * j);
      }
    }
  }
}

// Per scan tile and channel, the count of flagged entries (scan_passes(n) passes of STILE
// entries; the passes' loads are independent).
template <int C, class Src>
__global__ void __launch_bounds__(ST) k_scan_reduce(Src src, int64_t n, int32_t *tsum,
                                                    int64_t ntiles) {
  __shared__ int32_t sw[C][ST / 32];
  const int64_t tile = blockIdx.x;
  const int passes = scan_passes(n);
  int32_t cnt[C];
#pragma unroll
  for (int c = 0; c < C; ++c) cnt[c] = 0;
  const int64_t t0 = tile * passes * STILE;
  if (!reduce_tile<C>(src, t0, std::min<int64_t>(n, t0 + (int64_t)passes * STILE), cnt)) {
#pragma unroll SR
    for (int r = 0; r < passes; ++r) {
      const int64_t i0 = (tile * passes + r) * STILE + (int64_t)threadIdx.x * SI;
      ItemOps<C, Src> it;
      it.load(src, i0, n, true);
      it.count(cnt);
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

// In-place exclusive scan of each channel's tile sums; totals[c] = channel total.  Thread t
// owns a run of consecutive tiles: it sums them, one block-wide scan gives the run's offset,
// and a second pass over the run writes the prefixes.
template <int C>
__global__ void __launch_bounds__(1024) k_scan_tiles(int32_t *tsum, int64_t ntiles,
                                                     int32_t *totals) {
  __shared__ int32_t sw[32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
  const int64_t b0 = (int64_t)threadIdx.x * per;
  const int64_t b1 = b0 + per < ntiles ? b0 + per : ntiles;
  for (int c = 0; c < C; ++c) {
    int32_t *t = tsum + c * ntiles;
    int32_t sum = 0;
    for (int64_t i = b0; i < b1; ++i) sum += t[i];
    int32_t incl = warp_incl_scan(sum);
    if (lane == 31) sw[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int32_t w = sw[lane];
      sw[lane] = warp_incl_scan(w) - w;
    }
    __syncthreads();
    int32_t run = incl - sum + sw[warp];
    for (int64_t i = b0; i < b1; ++i) {
      const int32_t v = t[i];
      t[i] = run;
      run += v;
    }
    if (threadIdx.x == blockDim.x - 1) totals[c] = run;
    __syncthreads();
  }
}

// A tile that the source and emitter can rank in a form of their own, faster than the passes
// below (FlagSrc + RankEmit: a tile of leaves only); returns whether it did.  Entries t0..t1-1.
template <int C, class Src, class Emit>
__device__ __forceinline__ bool emit_tile(const Src &, const Emit &, int64_t, int64_t,
                                          const int32_t *, int64_t, int64_t) {
  return false;
}

// The exclusive counts of every entry: the tile's offset (toff) carried over its passes, each
// pass a block-wide scan.  The next pass's flags are loaded before this pass's scan (their
// latency overlaps it), and with at most 3 channels the per-thread counts (at most SI = 8 each,
// at most 256 in a warp) are packed 10 bits per channel so that one warp scan serves them all.
template <int C, class Src, class Emit>
__global__ void __launch_bounds__(ST) k_scan_emit(Src src, Emit em, int64_t n,
                                                  const int32_t *toff, int64_t ntiles) {
  __shared__ int32_t sw[2][C][ST / 32 + 1];  // per warp exclusive offsets, then the pass total
  const int64_t tile = blockIdx.x;
  const int passes = scan_passes(n);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {
    const int64_t t0 = tile * passes * STILE;
    if (emit_tile<C>(src, em, t0, std::min<int64_t>(n, t0 + (int64_t)passes * STILE), toff,
                     ntiles, tile))
      return;
  }
  int32_t carry[C];
#pragma unroll
  for (int c = 0; c < C; ++c) carry[c] = toff[c * ntiles + tile];
  ItemOps<C, Src> nx;
  {
    const int64_t p0 = tile * passes * STILE;
    if (p0 < n) nx.load(src, p0 + (int64_t)threadIdx.x * SI, n, false);
  }
  for (int r = 0; r < passes; ++r) {
    const int64_t p0 = (tile * passes + r) * STILE;
    if (p0 >= n) break;  // the same for the whole CTA
    const int64_t i0 = p0 + (int64_t)threadIdx.x * SI;
    const ItemOps<C, Src> it = nx;
    if (r + 1 < passes && p0 + STILE < n) nx.load(src, p0 + STILE + (int64_t)threadIdx.x * SI, n, false);
    int32_t cnt[C];
#pragma unroll
    for (int c = 0; c < C; ++c) cnt[c] = 0;
    it.count(cnt);
    int32_t pre[C];
    int32_t (&w)[C][ST / 32 + 1] = sw[r & 1];
    if (C <= 3) {
      int32_t pk = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) pk |= cnt[c] << (10 * c);
      const int32_t incl = warp_incl_scan(pk);
      const int32_t ex = incl - pk;
#pragma unroll
      for (int c = 0; c < C; ++c) {
        pre[c] = (ex >> (10 * c)) & 1023;
        if (lane == 31) w[c][warp] = (incl >> (10 * c)) & 1023;
      }
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        int32_t incl = warp_incl_scan(cnt[c]);
        pre[c] = incl - cnt[c];
        if (lane == 31) w[c][warp] = incl;
      }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        int32_t v = lane < ST / 32 ? w[c][lane] : 0;
        int32_t sc = warp_incl_scan(v);
        if (lane < ST / 32) w[c][lane] = sc - v;
        if (lane == ST / 32 - 1) w[c][ST / 32] = sc;
      }
    }
    __syncthreads();
    int32_t run[C];
#pragma unroll
    for (int c = 0; c < C; ++c) run[c] = carry[c] + w[c][warp] + pre[c];
    it.emit(em, i0, n, run);
#pragma unroll
    for (int c = 0; c < C; ++c) carry[c] += w[c][ST / 32];
    // the next pass writes the other half of sw; the one after this half again, behind the
    // next pass's two barriers
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

// Runs reduce + tile scan; leaves the tile offsets in *d_scratch (caller frees), followed by
// the C channel totals, and copies the totals to h_totals (synchronising the stream); with
// h_totals null the totals stay on the device only and nothing waits.
template <int C, class Src>
int scan_prepare(const Src &src, int64_t n, cudaStream_t s, int32_t **d_scratch,
                 int64_t *ntiles_out, int32_t *h_totals, const int32_t *d_extra = nullptr,
                 int32_t *h_extra = nullptr) {
  const int64_t tile_n = (int64_t)STILE * scan_passes(n);
  const int64_t ntiles = (n + tile_n - 1) / tile_n;
  *ntiles_out = ntiles;
  *d_scratch = nullptr;
  int32_t *pin = pinned_counts();
  if (!pin) {
    set_error("cudaHostAlloc of the count staging buffer failed");
    return VX_ENOMEM;
  }
  if (ntiles == 0) {
    if (h_totals)
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
  if (!h_totals) return VX_OK;
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
  if (tm && tm->on) VX_CHECK(tm->begin(KK_CSF_BUILD, n * k * 4));  // + the arrays, below
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
    if (tm && tm->on)
      for (int d = 0; d < k; ++d) tm->add_work(N[d] * (4 + (d > 0 ? 4 : 0) + (d + 1 < k ? 4 : 0)));
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
  // the segments are in depth order, so the depth is the number of segment starts <= i
  __device__ int depth_of(int64_t i) const {
    int d = 0;
#pragma unroll
    for (int e = 1; e < VX_KMAX; ++e) d += (e < sg.k && i >= sg.off[e]) ? 1 : 0;
    return d;
  }
  __device__ unsigned flags(int64_t i, bool) const {
    return f[i] ? (1u << depth_of(i)) : 0u;
  }
};

// the eight flags of a thread in one 8-byte load (the array is 256-byte aligned, i0 % 8 == 0)
__device__ __forceinline__ void load_items(const FlagSrc &src, int64_t i0, int64_t n, bool,
                                           unsigned (&m)[SI]) {
  static_assert(SI == 8, "one 8-byte load per thread");
  if (i0 + SI <= n) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(src.f + i0));
    const int d0 = src.depth_of(i0), d1 = src.depth_of(i0 + SI - 1);
#pragma unroll
    for (int j = 0; j < SI; ++j) {
      const unsigned b = ((j < 4 ? v.x : v.y) >> (8 * (j & 3))) & 0xffu;
      const int d = d0 == d1 ? d0 : src.depth_of(i0 + j);
      m[j] = b ? (1u << d) : 0u;
    }
  } else {
#pragma unroll
    for (int j = 0; j < SI; ++j) m[j] = i0 + j < n ? src.flags(i0 + j, false) : 0u;
  }
}

// A tile of leaves only (the last segment): 32 flag bytes (0 or 1 each) per thread and step.
template <int C>
__device__ __forceinline__ bool reduce_tile(const FlagSrc &src, int64_t t0, int64_t t1,
                                            int32_t (&cnt)[C]) {
  if (t0 < src.sg.off[C - 1]) return false;  // the same for the whole CTA
  int32_t c = 0;
  for (int64_t e0 = t0 + (int64_t)threadIdx.x * 32; e0 < t1; e0 += (int64_t)ST * 32) {
    uint32_t nz[8];
    nonzero32(src.f, e0, t1, nz);
#pragma unroll
    for (int q = 0; q < 8; ++q) c += __popc(nz[q]);
  }
  cnt[C - 1] += c;
  return true;
}

// The ranks of a pruned tree: rank[i] (the kept nodes of its depth before node i) for the inner
// depths (i < loff, the leaf segment's start), and for the leaf depth one count per aligned
// 8-entry word of the flag array, rank8[w - w0] = the kept leaves before word w; a leaf's rank
// is its word's count plus the kept leaves before it in the word (a popcount of the word's flag
// bytes, 0 or 1 each).  Half a byte per leaf is written and read instead of four.
struct RankView {
  const int32_t *rank;
  const int32_t *rank8;
  const uint8_t *flags;
  int64_t loff, w0;
  __device__ __forceinline__ int32_t at(int64_t i) const {
    if (i < loff) return __ldg(rank + i);
    const int64_t b = i & ~(int64_t)7;
    const uint64_t v = __ldg(reinterpret_cast<const unsigned long long *>(flags + b));
    const int hi = (int)(i - b), lo = loff > b ? (int)(loff - b) : 0;  // lo <= hi < 8
    uint64_t m = hi == 0 ? 0ull : (~0ull >> (64 - 8 * hi));            // bytes [0, hi)
    m &= ~0ull << (8 * lo);                                            // and >= loff
    return __ldg(rank8 + ((b >> 3) - w0)) + __popcll(v & m);
  }
  // The kept nodes of one depth (its segment starting at lo) before the absolute index a, a
  // multiple of 32 with a > lo - 32: zero before the segment, else an inner rank or, in the
  // leaf segment, the count of a's word (a is 8-aligned).  The lanes of a warp that read it
  // for one window read the same entry.
  __device__ __forceinline__ int32_t base32(int64_t a, int64_t lo) const {
    if (a < lo) return 0;
    return a < loff ? __ldg(rank + a) : __ldg(rank8 + ((a >> 3) - w0));
  }
};

// A warp's window of 32 consecutive absolute indices a .. a+31 (a a multiple of 32) over one
// depth's segment [lo, hi): the lane's node is a + lane; each kept node's rank is the window's
// base (RankView::base32) plus the kept lanes below it in the warp's ballot.
__device__ __forceinline__ int32_t window_rank(int32_t base, unsigned bal) {
  return base + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
}

struct RankEmit {
  int32_t *rank, *rank8;
  int64_t loff, w0;
  FlagSrc src;
  __device__ void operator()(int64_t i, unsigned m, const int32_t *excl) const {
    if (i < loff) rank[i] = excl[src.depth_of(i)];
  }
  // a word holding leaves gets the leaf channel's count at its start (for the word where the
  // leaf segment begins, no leaf lies before it, so the count is the leaves' first rank)
  template <int C>
  __device__ __forceinline__ void word(int64_t i0, const int32_t (&run)[C]) const {
    if (i0 + SI > loff) rank8[(i0 >> 3) - w0] = run[C - 1];
  }
};

// the eight ranks of a thread: two 16-byte stores for inner nodes (rank is 256-byte aligned),
// the word's count where it holds leaves
template <int C>
__device__ __forceinline__ void emit_items(const RankEmit &em, int64_t i0, int64_t n,
                                           const unsigned (&m)[SI], int32_t (&run)[C]) {
  if (i0 < n) em.word<C>(i0, run);
  if (i0 + SI <= n && i0 + SI <= em.loff) {
    int32_t r[SI];
    const int d0 = em.src.depth_of(i0), d1 = em.src.depth_of(i0 + SI - 1);
#pragma unroll
    for (int j = 0; j < SI; ++j) {
      const int dj = d0 == d1 ? d0 : em.src.depth_of(i0 + j);
      int32_t v = 0;
#pragma unroll
      for (int c = 0; c < C; ++c) v = c == dj ? run[c] : v;
      r[j] = v;
#pragma unroll
      for (int c = 0; c < C; ++c) run[c] += (m[j] >> c) & 1u;
    }
    int4 *dst = reinterpret_cast<int4 *>(em.rank + i0);
    dst[0] = make_int4(r[0], r[1], r[2], r[3]);
    dst[1] = make_int4(r[4], r[5], r[6], r[7]);
  } else {
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
}

// A tile of leaves only: their ranks are one count per 8-entry word, so a thread takes four
// words (32 flag bytes, two 16-byte loads) per step and one block-wide scan serves 8192
// entries, against 2048 per pass of the general form (whose barriers bound the scan).
template <int C>
__device__ __forceinline__ bool emit_tile(const FlagSrc &src, const RankEmit &em, int64_t t0,
                                          int64_t t1, const int32_t *toff, int64_t ntiles,
                                          int64_t tile) {
  if (t0 < em.loff) return false;  // the same for the whole CTA
  constexpr int WPT = 4;
  __shared__ int32_t s_w[ST / 32 + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t carry = toff[(C - 1) * ntiles + tile];
  for (int64_t b = t0; b < t1; b += (int64_t)ST * WPT * 8) {
    const int64_t e0 = b + (int64_t)threadIdx.x * WPT * 8;  // a multiple of 32
    int32_t c[WPT];
    if (e0 + WPT * 8 <= t1) {
      const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(src.f + e0));
      const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(src.f + e0 + 16));
      c[0] = __popc(v0.x) + __popc(v0.y);
      c[1] = __popc(v0.z) + __popc(v0.w);
      c[2] = __popc(v1.x) + __popc(v1.y);
      c[3] = __popc(v1.z) + __popc(v1.w);
    } else {
#pragma unroll
      for (int j = 0; j < WPT; ++j) {
        c[j] = 0;
        for (int q = 0; q < 8; ++q) {
          const int64_t i = e0 + 8 * j + q;
          if (i < t1) c[j] += src.f[i] ? 1 : 0;
        }
      }
    }
    const int32_t sum = c[0] + c[1] + c[2] + c[3];
    const int32_t incl = warp_incl_scan(sum);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int32_t v = lane < ST / 32 ? s_w[lane] : 0;
      const int32_t sc = warp_incl_scan(v);
      if (lane < ST / 32) s_w[lane] = sc - v;
      if (lane == ST / 32 - 1) s_w[ST / 32] = sc;
    }
    __syncthreads();
    int32_t run = carry + s_w[warp] + incl - sum;
#pragma unroll
    for (int j = 0; j < WPT; ++j) {
      if (e0 + 8 * j < t1) em.rank8[((e0 >> 3) + j) - em.w0] = run;
      run += c[j];
    }
    carry += s_w[ST / 32];
    __syncthreads();  // s_w is rewritten by the next step
  }
  return true;
}

// FlagSrc: the eight flag bytes of a thread (0 or 1 each) usually lie in one depth's segment;
// then their count is the popcount of the two words and their exclusive ranks are the byte-wise
// prefix sums (w * 0x01010101 holds the inclusive ones, at most 4 per byte: no carries).
template <int C>
struct ItemOps<C, FlagSrc> {
  uint2 v;
  int d;           // the depth of all eight entries, or -1 (another form: m)
  unsigned m[SI];  // per-entry channel bits when d < 0
  __device__ __forceinline__ void load(const FlagSrc &src, int64_t i0, int64_t n, bool) {
    d = -1;
    v = make_uint2(0u, 0u);
    if (i0 + SI <= n) {
      v = __ldg(reinterpret_cast<const uint2 *>(src.f + i0));
      const int d0 = src.depth_of(i0), d1 = src.depth_of(i0 + SI - 1);
      if (d0 == d1) {
        d = d0;
        return;
      }
    }
    load_items(src, i0, n, false, m);
  }
  __device__ __forceinline__ void count(int32_t (&cnt)[C]) const {
    if (d >= 0) {
      const int32_t pc = __popc(v.x) + __popc(v.y);
#pragma unroll
      for (int c = 0; c < C; ++c) cnt[c] += c == d ? pc : 0;
    } else {
#pragma unroll
      for (int j = 0; j < SI; ++j)
#pragma unroll
        for (int c = 0; c < C; ++c) cnt[c] += (m[j] >> c) & 1u;
    }
  }
  __device__ __forceinline__ void emit(const RankEmit &em, int64_t i0, int64_t n,
                                       int32_t (&run)[C]) const {
    if (d < 0) {
      emit_items<C>(em, i0, n, m, run);
      return;
    }
    int32_t base = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) base = c == d ? run[c] : base;
    if (d == C - 1) {  // eight leaves: their word's count only
      em.word<C>(i0, run);
      run[C - 1] += __popc(v.x) + __popc(v.y);
      return;
    }
    const uint32_t px = v.x * 0x01010101u, py = v.y * 0x01010101u;
    const uint32_t ex = px - v.x, ey = py - v.y;
    const int32_t tx = (int32_t)(px >> 24), ty = (int32_t)(py >> 24);
    int4 *dst = reinterpret_cast<int4 *>(em.rank + i0);
    dst[0] = make_int4(base + (int32_t)(ex & 0xffu), base + (int32_t)((ex >> 8) & 0xffu),
                       base + (int32_t)((ex >> 16) & 0xffu), base + (int32_t)(ex >> 24));
    const int32_t b1 = base + tx;
    dst[1] = make_int4(b1 + (int32_t)(ey & 0xffu), b1 + (int32_t)((ey >> 8) & 0xffu),
                       b1 + (int32_t)((ey >> 16) & 0xffu), b1 + (int32_t)(ey >> 24));
#pragma unroll
    for (int c = 0; c < C; ++c) run[c] += c == d ? tx + ty : 0;
  }
};

// Flags of depth d from those of depth d+1: node p is kept iff one of its children
// ptr[p] .. ptr[p+1]-1 (at flags[coff + child]) is.  Three forms, by the mean number of
// children per node.  flags is 256-byte aligned and has 16 bytes of padding after its last
// entry for the loads that run past a range's end.
//
// Long child ranges: one warp per node; each lane tests 16 flags per 16-byte load (512 per
// warp step, from the 16-byte boundary below the range) and the warp stops at the first step
// holding a kept child.
__global__ void k_mark_parents(const int32_t *__restrict__ ptr, int64_t n,
                               const uint8_t *__restrict__ flags, int64_t coff,
                               uint8_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n; p += nw) {
    const int64_t lo = coff + __ldg(ptr + p), hi = coff + __ldg(ptr + p + 1);
    bool any = false;
    for (int64_t b = lo & ~(int64_t)15; b < hi; b += 512) {  // the same trip count for all lanes
      const int64_t c = b + 16 * lane;
      bool hit = false;
      if (c < hi) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(flags + c));
        // the bytes [s, e) of the 16 loaded lie in the child range; two 8-byte halves, each
        // masked to its part of the range
        const int s = lo > c ? (int)(lo - c) : 0, e = hi < c + 16 ? (int)(hi - c) : 16;
        const uint64_t w[2] = {(uint64_t)v.x | ((uint64_t)v.y << 32),
                               (uint64_t)v.z | ((uint64_t)v.w << 32)};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int sh = s - 8 * h < 0 ? 0 : (s - 8 * h > 8 ? 8 : s - 8 * h);
          const int eh = e - 8 * h < 0 ? 0 : (e - 8 * h > 8 ? 8 : e - 8 * h);
          const int width = eh > sh ? eh - sh : 0;
          const uint64_t m =
              width <= 0 ? 0ull : (width >= 8 ? ~0ull : ((1ull << (8 * width)) - 1ull)) << (8 * sh);
          hit = hit || (w[h] & m) != 0ull;
        }
      }
      if (__any_sync(0xffffffffu, hit)) {
        any = true;
        break;
      }
    }
    if (lane == 0) out[p] = any ? 1 : 0;
  }
}


// Whether the flag bytes [lo, hi) that fall in the 16 bytes v (loaded from c, 16-aligned)
// hold a kept child.
__device__ __forceinline__ bool block_hit(const uint4 v, int64_t c, int64_t lo, int64_t hi) {
  const int s = lo > c ? (int)(lo - c) : 0, e = hi < c + 16 ? (int)(hi - c) : 16;
  const uint64_t w[2] = {(uint64_t)v.x | ((uint64_t)v.y << 32), (uint64_t)v.z | ((uint64_t)v.w << 32)};
  bool hit = false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int sh = s - 8 * h < 0 ? 0 : (s - 8 * h > 8 ? 8 : s - 8 * h);
    const int eh = e - 8 * h < 0 ? 0 : (e - 8 * h > 8 ? 8 : e - 8 * h);
    const int width = eh > sh ? eh - sh : 0;
    const uint64_t m =
        width <= 0 ? 0ull : (width >= 8 ? ~0ull : ((1ull << (8 * width)) - 1ull)) << (8 * sh);
    hit = hit || (w[h] & m) != 0ull;
  }
  return hit;
}

// Long child ranges on many nodes: one thread per node, 32 flag bytes per step (two 16-byte
// loads from the 16-byte boundary below its range), stopping at the first kept child, which
// a node with many kept children finds in its first step; the warp-per-node form spent a
// warp's sequence of dependent loads on every node in turn.
__global__ void k_mark_parents_l(const int32_t *__restrict__ ptr, int64_t n,
                                 const uint8_t *__restrict__ flags, int64_t coff,
                                 uint8_t *__restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = coff + __ldg(ptr + p), hi = coff + __ldg(ptr + p + 1);
    bool any = false;
    for (int64_t b = lo & ~(int64_t)15; b < hi && !any; b += 32) {
      const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(flags + b));
      const uint4 v1 = b + 16 < hi ? __ldg(reinterpret_cast<const uint4 *>(flags + b + 16))
                                   : make_uint4(0u, 0u, 0u, 0u);
      any = block_hit(v0, b, lo, hi) || (b + 16 < hi && block_hit(v1, b + 16, lo, hi));
    }
    out[p] = any ? 1 : 0;
  }
}

// Short child ranges (a few children per node, as in the trees of small systems): one thread
// per node, eight flag bytes per load from the 8-byte boundary below its
// range (the 16 bytes of padding after the flags cover the last load).
__global__ void k_mark_parents_t(const int32_t *__restrict__ ptr, int64_t n,
                                 const uint8_t *__restrict__ flags, int64_t coff,
                                 uint8_t *__restrict__ out) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = coff + __ldg(ptr + p), hi = coff + __ldg(ptr + p + 1);
    bool any = false;
    for (int64_t b = lo & ~(int64_t)7; b < hi && !any; b += 8) {
      const uint64_t w = __ldg(reinterpret_cast<const unsigned long long *>(flags + b));
      const int sh = lo > b ? (int)(lo - b) : 0, eh = hi < b + 8 ? (int)(hi - b) : 8;
      const int width = eh - sh;  // >= 1: b < hi and b + 8 > lo
      const uint64_t m = (width >= 8 ? ~0ull : ((1ull << (8 * width)) - 1ull)) << (8 * sh);
      any = (w & m) != 0ull;
    }
    out[p] = any ? 1 : 0;
  }
}

// Child ranges of moderate length: from the children's side, out (zeroed before) gets 1 at the parent of every kept child.  Thread = one 16-byte
// block of the flag array (absolute offsets, so the loads are aligned) over the children's
// range [cs, ce); a block with a kept child reads those children's parent indices.  Several
// threads may store the same 1 to one parent's byte.
__global__ void k_mark_parents_s(const int32_t *__restrict__ cpar, int64_t cs, int64_t ce,
                                 const uint8_t *__restrict__ flags, uint8_t *__restrict__ out) {
  const int64_t q0 = cs >> 4, q1 = (ce + 15) >> 4;
  for (int64_t q = q0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < q1;
       q += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(flags) + q);
    if ((v.x | v.y | v.z | v.w) == 0u) continue;
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int64_t a = 16 * q + j;
      if (a < cs || a >= ce || ((w[j >> 2] >> (8 * (j & 3))) & 0xffu) == 0u) continue;
      out[__ldg(cpar + (a - cs))] = 1;
    }
  }
}

// kptr[d][g_d(p)] = rank of the first kept child of kept node p (depth d < k-1)
template <int D>
__global__ void k_kptr(CsfView c, const uint8_t *__restrict__ flags, const RankView rank,
                       Segs sg, int32_t *kptr) {
  constexpr int d = D;
  const int64_t lo = sg.off[d], hi = lo + c.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // a warp takes a 32-aligned window of the flag array (blockDim and stride multiples of 32)
  for (int64_t a = (lo & ~(int64_t)31) + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
       a < hi; a += stride) {
    const int64_t i = a + (threadIdx.x & 31);
    const bool kept = i >= lo && i < hi && flags[i];
    const int32_t base = rank.base32(a, lo);
    const unsigned bal = __ballot_sync(0xffffffffu, kept);
    if (kept) kptr[window_rank(base, bal)] = rank.at(sg.off[d + 1] + c.ptr[d][i - lo]);
  }
}

struct KptrSet {
  const int32_t *k[VX_KMAX];  // kptr[d], n_d + 1 entries (last = n_{d+1})
};

__device__ __forceinline__ int32_t chain(const KptrSet &K, int a, int t, int32_t r) {
#pragma unroll
  for (int e = 0; e < VX_KMAX; ++e)
    if (e >= a && e < t) r = K.k[e][r];
  return r;
}

// Bisection of depth d: every kept depth-d node writes its 2^(d+1) copies.  k and d are
// template arguments so that the path arrays stay in registers.  Per kept node, the plan of
// its copies (split_plan: loads only) and then their stores (split_write): copies b and b+1
// (b even) are neighbours (idx even), so each pair is one 8-byte store per array.
struct SplitPlan {
  int64_t bd, bm, bp;
  int64_t Dd[VX_KMAX], Dm[VX_KMAX], Dp[VX_KMAX];
  int32_t lab2;
};

template <int KK, int D>
__device__ __forceinline__ void split_plan(const CsfView &in, const RankView &rank,
                                           const Segs &sg, const KptrSet &K, int64_t p,
                                           int32_t gd, SplitPlan &P) {
  constexpr int k = KK, d = D;
  int64_t path[VX_KMAX];
  int32_t g[VX_KMAX];
  path[d] = p;
#pragma unroll
  for (int a = d; a > 0; --a) path[a - 1] = __ldg(in.par[a] + path[a]);
#pragma unroll
  for (int a = 0; a < d; ++a) g[a] = rank.at(sg.off[a] + path[a]);
  g[d] = gd;
  // F_t(p_a) and D_t(p_a) for t = d-1, d, d+1
  P.bd = P.bm = P.bp = 0;
  int64_t prevF_d = 0, prevF_m = 0, prevF_p = 0;
#pragma unroll
  for (int a = 0; a <= d; ++a) {
    const int64_t Fd = chain(K, a, d, g[a]);
    P.Dd[a] = chain(K, a, d, g[a] + 1) - Fd;
    P.bd += (Fd - prevF_d) << (d - a + 1);
    prevF_d = Fd;
    if (a < d) {
      const int64_t Fm = chain(K, a, d - 1, g[a]);
      P.Dm[a] = chain(K, a, d - 1, g[a] + 1) - Fm;
      P.bm += (Fm - prevF_m) << (d - a);
      prevF_m = Fm;
    }
    if (d + 1 < k) {
      const int64_t Fp = chain(K, a, d + 1, g[a]);
      P.Dp[a] = chain(K, a, d + 1, g[a] + 1) - Fp;
      P.bp += (Fp - prevF_p) << (d - a + 2);
      prevF_p = Fp;
    }
  }
  P.lab2 = 2 * __ldg(in.lab[d] + p);
}

template <int KK, int D>
__device__ __forceinline__ void split_write(const CsfView &out, const SplitPlan &P) {
  constexpr int k = KK, d = D;
  const int nb = 1 << (d + 1);
  for (int b = 0; b < nb; b += 2) {
    // the copies b and b + 1 differ in the last bit only: idx + 1, the same parent, and the
    // child pointer moved by 2 D_{d+1}(p_d)
    int64_t idx = P.bd, pidx = P.bm, cidx = P.bp;
#pragma unroll
    for (int a = 0; a < d; ++a) {
      const int64_t bit = (b >> (d - a)) & 1;
      idx += bit * (P.Dd[a] << (d - a));
      pidx += bit * (P.Dm[a] << (d - 1 - a));
      if (d + 1 < k) cidx += bit * (P.Dp[a] << (d - a + 1));
    }
    *reinterpret_cast<int2 *>(out.lab[d] + idx) = make_int2(P.lab2, P.lab2 + 1);
    if (d > 0) *reinterpret_cast<int2 *>(out.par[d] + idx) = make_int2((int32_t)pidx, (int32_t)pidx);
    if (d + 1 < k)
      *reinterpret_cast<int2 *>(out.ptr[d] + idx) =
          make_int2((int32_t)cidx, (int32_t)(cidx + (P.Dp[d] << 1)));
  }
}

// A warp takes kSplitU consecutive 32-aligned windows of the flag array per step (blockDim
// and the stride multiples of 32): the plans of both windows' kept nodes (their loads) before
// any of their stores.
constexpr int kSplitU = 2;
template <int KK, int D>
__global__ void k_split(CsfView in, const uint8_t *__restrict__ flags, const RankView rank,
                        Segs sg, KptrSet K, CsfView out) {
  constexpr int d = D, U = kSplitU;
  const int64_t lo = sg.off[d], hi = lo + in.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * U;
  const int lane = threadIdx.x & 31;
  for (int64_t a = (lo & ~(int64_t)31) + ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * U;
       a < hi; a += stride) {
    bool kept[U];
    int32_t base[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = a + 32 * u + lane;
      kept[u] = i >= lo && i < hi && flags[i];
      base[u] = a + 32 * u < hi ? rank.base32(a + 32 * u, lo) : 0;
    }
    SplitPlan P[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned bal = __ballot_sync(0xffffffffu, kept[u]);
      if (kept[u])
        split_plan<KK, D>(in, rank, sg, K, a + 32 * u + lane - lo, window_rank(base[u], bal), P[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (kept[u]) split_write<KK, D>(out, P[u]);
  }
}

// Compaction of depth d: kept node p goes to its rank.  A warp takes kGatherU consecutive
// 32-aligned windows of the flag array per step (blockDim and the stride multiples of 32), so
// that the windows' flag, label, parent and rank loads are in flight together (one window per
// step left the kernel waiting on each kept node's chain of loads in turn).
constexpr int kGatherU = 4;
template <int D>
__global__ void k_gather(CsfView in, const uint8_t *__restrict__ flags, const RankView rank,
                         Segs sg, CsfView out, int32_t *index) {
  constexpr int d = D, U = kGatherU;
  const int64_t lo = sg.off[d], hi = lo + in.N[d];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x * U;
  const int lane = threadIdx.x & 31;
  for (int64_t a = (lo & ~(int64_t)31) + ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * U;
       a < hi; a += stride) {
    bool kept[U];
    int32_t base[U], lab[U], prank[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = a + 32 * u + lane;
      kept[u] = i >= lo && i < hi && flags[i];
      base[u] = a + 32 * u < hi ? rank.base32(a + 32 * u, lo) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = a + 32 * u + lane - lo;
      lab[u] = kept[u] ? __ldg(in.lab[d] + p) : 0;
      prank[u] = (d > 0 && kept[u]) ? __ldg(rank.rank + sg.off[d - 1] + __ldg(in.par[d] + p)) : 0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const unsigned bal = __ballot_sync(0xffffffffu, kept[u]);
      if (!kept[u]) continue;
      const int32_t r = window_rank(base[u], bal);
      const int64_t p = a + 32 * u + lane - lo;
      out.lab[d][r] = lab[u];
      if (d > 0) out.par[d][r] = prank[u];
      if (index && d == in.k - 1) index[r] = (int32_t)p;
    }
  }
}

// The leaf depth's compaction (k_gather<D>, D = k-1) that also writes each kept leaf's
// grid-index code (k_box_codes' formula, cb = 4 or 8 bytes) at its rank, for a destination
// across the host link (mapped pinned memory), where a partial cache line costs about as much
// as a full one: a CTA takes a contiguous chunk of kGatherChunk entries, stages the chunk's
// codes (consecutive ranks) in shared memory and writes them as whole aligned lines, only the
// chunk's two ends partial.
constexpr int kGatherChunk = 2048;
template <int D>
__global__ void __launch_bounds__(256)
    k_gather_codes(CsfView in, const uint8_t *__restrict__ flags, const RankView rank, Segs sg,
                   CsfView out, int32_t *index, void *codes, int cb) {
  constexpr int d = D;
  extern __shared__ __align__(16) unsigned char s_codes[];
  __shared__ int32_t s_cnt;
  const int64_t lo = sg.off[d], hi = lo + in.N[d];
  const int64_t a0 = lo & ~(int64_t)31;
  const int64_t nch = (hi - a0 + kGatherChunk - 1) / kGatherChunk;
  const int lane = threadIdx.x & 31;
  for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const int64_t A = a0 + ch * kGatherChunk;  // a multiple of 32, > lo - 32, < hi
    const int32_t R0 = rank.base32(A, lo);     // the chunk's first rank
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int64_t a = A + (threadIdx.x & ~31); a < A + kGatherChunk && a < hi; a += blockDim.x) {
      const int64_t i = a + lane, p = i - lo;
      const bool kept = i >= lo && i < hi && flags[i];
      const int32_t base = rank.base32(a, lo);
      const unsigned bal = __ballot_sync(0xffffffffu, kept);
      if (lane == 0 && bal) atomicAdd(&s_cnt, __popc(bal));
      if (!kept) continue;
      const int32_t r = window_rank(base, bal);
      const int32_t lab = __ldg(in.lab[d] + p);
      const int32_t pp = d > 0 ? __ldg(in.par[d] + p) : 0;
      out.lab[d][r] = lab;
      if (d > 0) out.par[d][r] = __ldg(rank.rank + sg.off[d - 1] + pp);
      if (index) index[r] = (int32_t)p;
      uint64_t code = (uint32_t)lab;
      int32_t q = pp;
#pragma unroll
      for (int e = d - 1; e >= 0; --e) {
        code |= (uint64_t)(uint32_t)__ldg(in.lab[e] + q) << (in.level * (d - e));
        if (e > 0) q = __ldg(in.par[e] + q);
      }
      if (cb == 4)
        reinterpret_cast<uint32_t *>(s_codes)[r - R0] = (uint32_t)code;
      else
        reinterpret_cast<uint64_t *>(s_codes)[r - R0] = code;
    }
    __syncthreads();
    // ranks R0 .. R0 + s_cnt - 1, written from the 32-aligned rank below R0: each warp store
    // covers whole lines
    const int64_t e0 = R0, e1 = (int64_t)R0 + s_cnt;
    for (int64_t g = (e0 & ~(int64_t)31) + threadIdx.x; g < e1; g += blockDim.x) {
      if (g < e0) continue;
      if (cb == 4)
        static_cast<uint32_t *>(codes)[g] = reinterpret_cast<const uint32_t *>(s_codes)[g - e0];
      else
        static_cast<uint64_t *>(codes)[g] = reinterpret_cast<const uint64_t *>(s_codes)[g - e0];
    }
    __syncthreads();  // s_codes and s_cnt are rewritten by the next chunk
  }
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sm_count() * 32) b = (int64_t)sm_count() * 32;
  if (b < 1) b = 1;
  return (int)b;
}

// Forest segments: seg_off[d * (S+1) + s] is the first depth-d node of tree-set s (s = 0..S,
// seg_off[.. + S] = N_d); kept[d * (S+1) + s] receives the kept depth-d nodes before it.
__global__ void k_seg_kept(const int64_t *__restrict__ seg_off, int S, int k,
                           const RankView rank, Segs sg, const int32_t *totals,
                           int64_t *__restrict__ kept) {
  const int64_t n = (int64_t)k * (S + 1);
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(j / (S + 1));
    const int64_t i = seg_off[j];
    kept[j] = i >= sg.off[d + 1] - sg.off[d] ? (int64_t)totals[d] : (int64_t)rank.at(sg.off[d] + i);
  }
}

// run-time depth -> template argument
void launch_kptr(int d, int blocks, cudaStream_t s, const CsfView &in, const uint8_t *flags,
                 const RankView &rank, const Segs &sg, int32_t *kptr) {
  switch (d) {
    case 0: k_kptr<0><<<blocks, 256, 0, s>>>(in, flags, rank, sg, kptr); break;
    case 1: k_kptr<1><<<blocks, 256, 0, s>>>(in, flags, rank, sg, kptr); break;
    case 2: k_kptr<2><<<blocks, 256, 0, s>>>(in, flags, rank, sg, kptr); break;
    case 3: k_kptr<3><<<blocks, 256, 0, s>>>(in, flags, rank, sg, kptr); break;
    default: k_kptr<4><<<blocks, 256, 0, s>>>(in, flags, rank, sg, kptr); break;
  }
}

void launch_gather(int d, int blocks, cudaStream_t s, const CsfView &in, const uint8_t *flags,
                   const RankView &rank, const Segs &sg, const CsfView &out, int32_t *index,
                   void *codes, int cb) {
  if (codes) {  // the leaf depth with its codes
    const int64_t nch = (in.N[d] + 31 + kGatherChunk - 1) / kGatherChunk;
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(nch, (int64_t)sm_count() * 8));
    const size_t sm = (size_t)kGatherChunk * cb;
    switch (d) {
      case 0: k_gather_codes<0><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
      case 1: k_gather_codes<1><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
      case 2: k_gather_codes<2><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
      case 3: k_gather_codes<3><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
      case 4: k_gather_codes<4><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
      default: k_gather_codes<5><<<g, 256, sm, s>>>(in, flags, rank, sg, out, index, codes, cb); break;
    }
    return;
  }
  switch (d) {
    case 0: k_gather<0><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
    case 1: k_gather<1><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
    case 2: k_gather<2><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
    case 3: k_gather<3><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
    case 4: k_gather<4><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
    default: k_gather<5><<<blocks, 256, 0, s>>>(in, flags, rank, sg, out, index); break;
  }
}

template <int KK>
void launch_split(int d, int blocks, cudaStream_t s, const CsfView &in, const uint8_t *flags,
                  const RankView &rank, const Segs &sg, const KptrSet &K, const CsfView &out) {
  switch (d) {
    case 0: k_split<KK, 0><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
    case 1: if (KK > 1) k_split<KK, (KK > 1 ? 1 : 0)><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
    case 2: if (KK > 2) k_split<KK, (KK > 2 ? 2 : 0)><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
    case 3: if (KK > 3) k_split<KK, (KK > 3 ? 3 : 0)><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
    case 4: if (KK > 4) k_split<KK, (KK > 4 ? 4 : 0)><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
    default: if (KK > 5) k_split<KK, (KK > 5 ? 5 : 0)><<<blocks, 256, 0, s>>>(in, flags, rank, sg, K, out); break;
  }
}

template <int C>
int prune_c(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
            cudaStream_t s, CsfObj *out, Timer *tm, const int64_t *d_seg_off = nullptr,
            int nseg = 0, int64_t *d_seg_kept = nullptr, int64_t cap = INT32_MAX,
            int64_t *h_seg_kept = nullptr, const CodesSink *sink = nullptr) {
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
    if (d_seg_kept)
      VX_CUDA(cudaMemsetAsync(d_seg_kept, 0, sizeof(int64_t) * (size_t)k * (nseg + 1), s));
    if (h_seg_kept)
      for (int64_t j = 0; j < (int64_t)k * (nseg + 1); ++j) h_seg_kept[j] = 0;
    return set_ptr_sentinels(out->v, s);
  }
  uint8_t *flags = nullptr;
  int32_t *rank = nullptr, *kptr = nullptr, *scratch = nullptr;
  int rc = VX_OK;
  // ranks: one per inner node, one per 8-entry word of the leaf segment (RankView)
  const int64_t loff = sg.off[k - 1], w0 = loff >> 3, nw8 = ((total - 1) >> 3) - w0 + 1;
  const int64_t rank_inner = (loff + 63) & ~(int64_t)63;  // rank8 256-byte aligned after it
  // algorithmic bytes: the leaves' keep flags and the inner ptr arrays read, one flag byte per
  // node and the ranks written
  int64_t prune_bytes = in.N[k - 1] + total + 4 * (loff + nw8);
  for (int d = 0; d + 1 < k; ++d) prune_bytes += 4 * (in.N[d] + 1);
  if (tm && tm->on) VX_CHECK(tm->begin(KK_PRUNE, prune_bytes));
  rc = dmalloc((void **)&flags, (size_t)total + 16, s);  // 16 bytes for the 16-byte loads
  if (rc == VX_OK) rc = dmalloc((void **)&rank, (size_t)(rank_inner + nw8) * sizeof(int32_t), s);
  const RankView rv{rank, rank + rank_inner, flags, loff, w0};
  if (rc == VX_OK) {
    cudaError_t e = cudaMemcpyAsync(flags + sg.off[k - 1], d_keep, (size_t)in.N[k - 1],
                                    cudaMemcpyDeviceToDevice, s);
    for (int d = k - 2; d >= 0 && e == cudaSuccess; --d) {
      if (in.N[d + 1] <= 32 * in.N[d]) {  // short child ranges: one thread per node
        int64_t blocks = (in.N[d] + 255) / 256;
        if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
        if (blocks < 1) blocks = 1;
        k_mark_parents_t<<<(unsigned)blocks, 256, 0, s>>>(in.ptr[d], in.N[d], flags,
                                                         sg.off[d + 1], flags + sg.off[d]);
      } else if (in.N[d + 1] > 128 * in.N[d]) {
        // long ranges: one thread per node where the nodes fill the GPU with threads, else one
        // warp per node
        if (in.N[d] >= (int64_t)sm_count() * 512) {
          int64_t blocks = (in.N[d] + 255) / 256;
          if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
          k_mark_parents_l<<<(unsigned)blocks, 256, 0, s>>>(in.ptr[d], in.N[d], flags,
                                                           sg.off[d + 1], flags + sg.off[d]);
        } else {
          int64_t blocks = (in.N[d] + 7) / 8;  // 8 warps per block
          if (blocks > (int64_t)sm_count() * 16) blocks = (int64_t)sm_count() * 16;
          if (blocks < 1) blocks = 1;
          k_mark_parents<<<(unsigned)blocks, 256, 0, s>>>(in.ptr[d], in.N[d], flags,
                                                         sg.off[d + 1], flags + sg.off[d]);
        }
      } else {  // scatter from the kept children to their parents
        e = cudaMemsetAsync(flags + sg.off[d], 0, (size_t)in.N[d], s);
        if (e != cudaSuccess) break;
        int64_t blocks = ((in.N[d + 1] + 31) / 16 + 255) / 256;
        if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
        if (blocks < 1) blocks = 1;
        k_mark_parents_s<<<(unsigned)blocks, 256, 0, s>>>(in.par[d + 1], sg.off[d + 1],
                                                         sg.off[d + 1] + in.N[d + 1], flags,
                                                         flags + sg.off[d]);
      }
      note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      set_error("marking kept nodes failed: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  FlagSrc src{flags, sg};
  int64_t ntiles = 0;
  int32_t nk[C];
  // with per-segment counts for the host, the channel totals and those counts travel back
  // together after the ranks (one wait instead of two)
  const bool one_wait = d_seg_off && h_seg_kept;
  if (rc == VX_OK) rc = scan_prepare<C>(src, total, s, &scratch, &ntiles, one_wait ? nullptr : nk);
  if (rc == VX_OK)
    rc = scan_emit<C>(src, RankEmit{rank, rank + rank_inner, loff, w0, src}, total, scratch,
                      ntiles, s);
  if (rc == VX_OK && d_seg_off) {
    // the channel totals sit after the tile sums in the scan scratch
    k_seg_kept<<<blocks_for((int64_t)k * (nseg + 1)), 256, 0, s>>>(
        d_seg_off, nseg, k, rv, sg, scratch + (int64_t)C * ntiles, d_seg_kept);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) {
      set_error("segment count kernel launch failed");
      rc = VX_ECUDA;
    }
  }
  if (rc == VX_OK && one_wait) {
    int32_t *pin = pinned_counts();
    cudaError_t e = cudaMemcpyAsync(pin, scratch + (int64_t)C * ntiles, C * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h_seg_kept, d_seg_kept, sizeof(int64_t) * (size_t)k * (nseg + 1),
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("reading the kept counts failed: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    } else {
      for (int c = 0; c < C; ++c) nk[c] = pin[c];
    }
  }
  // kept-tree first-child pointers
  KptrSet K{};
  int64_t koff[VX_KMAX + 1] = {0};
  for (int d = 0; d + 1 < k; ++d) koff[d + 1] = koff[d] + nk[d] + 1;
  int64_t newN[VX_KMAX] = {0};
  if (rc == VX_OK) {
    for (int d = 0; d < k; ++d) {
      newN[d] = split ? ((int64_t)nk[d] << (d + 1)) : nk[d];
      if (newN[d] > INT32_MAX || newN[d] > cap) {
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
  // algorithmic bytes: flags and ranks of every node read; per kept node its label, parent
  // (depth > 0) and child pointer (depth < k-1) read; the same arrays written per new node (a
  // split) or per kept node (a compaction)
  int64_t rebuild_bytes = total + 4 * (loff + nw8);
  for (int d = 0; d < k; ++d) {
    const int64_t w = 4 + (d > 0 ? 4 : 0) + (d + 1 < k ? 4 : 0);
    rebuild_bytes += ((int64_t)nk[d] + (split ? newN[d] : (int64_t)nk[d])) * w;
  }
  if (!split && d_index) rebuild_bytes += 4 * (int64_t)nk[k - 1];
  // a compaction's leaf codes, where the caller takes them now
  void *codes = nullptr;
  const int cb = k * in.level <= 32 ? 4 : 8;
  if (rc == VX_OK && !split && sink && nk[k - 1] > 0)
    rc = sink->get(sink->ctx, nk[k - 1], cb, &codes);
  if (rc == VX_OK && tm && tm->on) rc = tm->begin(split ? KK_SPLIT : KK_COMPACT, rebuild_bytes);
  for (int d = 0; d + 1 < k && rc == VX_OK; ++d) {
    launch_kptr(d, blocks_for(in.N[d]), s, in, flags, rv, sg, (int32_t *)K.k[d]);
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
      launch_split<C>(d, blocks_for(in.N[d]), s, in, flags, rv, sg, K, out->v);
    else
      launch_gather(d, blocks_for(in.N[d]), s, in, flags, rv, sg, out->v, d_index,
                    d == k - 1 ? codes : nullptr, cb);
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

// Each leaf's box as its index in the level's full grid, x_1 most significant:
// code = sum_d t_d << (level (k-1-d)); 4 bytes per code when k level <= 32, else 8.
template <typename C>
__global__ void k_box_codes(CsfView c, C *out) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int64_t p = i;
    uint64_t code = 0;
    for (int d = k - 1; d >= 0; --d) {
      code |= (uint64_t)(uint32_t)c.lab[d][p] << (c.level * (k - 1 - d));
      if (d > 0) p = c.par[d][p];
    }
    out[i] = (C)code;
  }
}

// indices of the nonzero bytes, in increasing order
struct ByteFlagSrc {
  const uint8_t *f;
  __device__ unsigned flags(int64_t i, bool) const { return f[i] ? 1u : 0u; }
};

// the eight flags of a thread in one 8-byte load where the address allows it
__device__ __forceinline__ void load_items(const ByteFlagSrc &src, int64_t i0, int64_t n, bool,
                                           unsigned (&m)[SI]) {
  static_assert(SI == 8, "one 8-byte load per thread");
  if (i0 + SI <= n && (reinterpret_cast<uintptr_t>(src.f + i0) & 7u) == 0) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(src.f + i0));
#pragma unroll
    for (int j = 0; j < SI; ++j) m[j] = (((j < 4 ? v.x : v.y) >> (8 * (j & 3))) & 0xffu) ? 1u : 0u;
  } else {
#pragma unroll
    for (int j = 0; j < SI; ++j) m[j] = i0 + j < n ? src.flags(i0 + j, false) : 0u;
  }
}
struct IndexEmit {
  int32_t *idx;
  __device__ void operator()(int64_t i, unsigned m, const int32_t *excl) const {
    if (m) idx[excl[0]] = (int32_t)i;
  }
};

// the nonzero bytes of a 32-bit word, as its bits 7, 15, 23 and 31
__device__ __forceinline__ uint32_t nonzero_bytes(uint32_t x) {
  return (((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x) & 0x80808080u;
}

// Sparse byte flags (a few selected among many): eight flags counted per 8-byte word, and a
// word without a flag emits nothing.
template <>
struct ItemOps<1, ByteFlagSrc> {
  uint2 v;
  bool word;       // v holds the eight flags
  unsigned m[SI];  // else the per-entry flags
  __device__ __forceinline__ void load(const ByteFlagSrc &src, int64_t i0, int64_t n, bool) {
    word = i0 + SI <= n && (reinterpret_cast<uintptr_t>(src.f + i0) & 7u) == 0;
    if (word) {
      v = __ldg(reinterpret_cast<const uint2 *>(src.f + i0));
      v = make_uint2(nonzero_bytes(v.x), nonzero_bytes(v.y));
    } else {
      load_items(src, i0, n, false, m);
    }
  }
  __device__ __forceinline__ void count(int32_t (&cnt)[1]) const {
    if (word) {
      cnt[0] += __popc(v.x) + __popc(v.y);
    } else {
#pragma unroll
      for (int j = 0; j < SI; ++j) cnt[0] += m[j] & 1u;
    }
  }
  template <class Emit>
  __device__ __forceinline__ void emit(const Emit &em, int64_t i0, int64_t n,
                                       int32_t (&run)[1]) const {
    if (!word) {
      emit_items<1>(em, i0, n, m, run);
      return;
    }
    if ((v.x | v.y) == 0u) return;
#pragma unroll
    for (int j = 0; j < SI; ++j) {
      const unsigned b = ((j < 4 ? v.x : v.y) >> (8 * (j & 3) + 7)) & 1u;
      if (b) {
        em(i0 + j, 1u, run);
        run[0] += 1;
      }
    }
  }
};

// Byte flags at a 16-byte aligned address: 32 per thread and step, counted by popcount; the
// emit scans a step only where a flag is set (a few selected among many).
template <int C>
__device__ __forceinline__ bool reduce_tile(const ByteFlagSrc &src, int64_t t0, int64_t t1,
                                            int32_t (&cnt)[C]) {
  if (reinterpret_cast<uintptr_t>(src.f) & 15u) return false;
  int32_t c = 0;
  for (int64_t e0 = t0 + (int64_t)threadIdx.x * 32; e0 < t1; e0 += (int64_t)ST * 32) {
    uint32_t nz[8];
    nonzero32(src.f, e0, t1, nz);
#pragma unroll
    for (int q = 0; q < 8; ++q) c += __popc(nz[q]);
  }
  cnt[0] += c;
  return true;
}

template <int C>
__device__ __forceinline__ bool emit_tile(const ByteFlagSrc &src, const IndexEmit &em, int64_t t0,
                                          int64_t t1, const int32_t *toff, int64_t ntiles,
                                          int64_t tile) {
  if (reinterpret_cast<uintptr_t>(src.f) & 15u) return false;
  __shared__ int32_t s_w[ST / 32 + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t carry = toff[tile];
  for (int64_t b = t0; b < t1; b += (int64_t)ST * 32) {
    const int64_t e0 = b + (int64_t)threadIdx.x * 32;
    uint32_t nz[8];
    int32_t sum = 0;
    if (e0 < t1) {
      nonzero32(src.f, e0, t1, nz);
#pragma unroll
      for (int q = 0; q < 8; ++q) sum += __popc(nz[q]);
    }
    if (!__syncthreads_or(sum)) continue;  // no flag in the step: nothing to emit
    const int32_t incl = warp_incl_scan(sum);
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int32_t v = lane < ST / 32 ? s_w[lane] : 0;
      const int32_t sc = warp_incl_scan(v);
      if (lane < ST / 32) s_w[lane] = sc - v;
      if (lane == ST / 32 - 1) s_w[ST / 32] = sc;
    }
    __syncthreads();
    int32_t run = carry + s_w[warp] + incl - sum;
    if (sum) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t bits = nz[q];
        while (bits) {
          const int j = (__ffs(bits) - 1) >> 3;
          em.idx[run++] = (int32_t)(e0 + 4 * q + j);
          bits &= bits - 1u;
        }
      }
    }
    carry += s_w[ST / 32];
    __syncthreads();  // s_w is rewritten by the next step
  }
  return true;
}

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
    case 4: return build_c<4>(k, level, d_tuples, n, s, out, tm);
    case 5: return build_c<5>(k, level, d_tuples, n, s, out, tm);
    default: return build_c<6>(k, level, d_tuples, n, s, out, tm);
  }
}

int csf_prune(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
              cudaStream_t s, CsfObj *out, Timer *tm, int64_t cap, const CodesSink *sink) {
  switch (in.k) {
    case 1: return prune_c<1>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
    case 2: return prune_c<2>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
    case 3: return prune_c<3>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
    case 4: return prune_c<4>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
    case 5: return prune_c<5>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
    default: return prune_c<6>(in, d_keep, split, d_index, s, out, tm, nullptr, 0, nullptr, cap, nullptr, sink);
  }
}

namespace {

// the depth-0 ancestor of leaf i
__device__ __forceinline__ int64_t root_of(const CsfView &c, int64_t i) {
  int64_t p = i;
  for (int d = c.k - 1; d > 0; --d) p = c.par[d][p];
  return p;
}

__global__ void k_root_counts(CsfView c, const uint8_t *__restrict__ keep,
                              unsigned long long *cnt) {
  const int64_t n = c.N[c.k - 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (keep[i]) atomicAdd(cnt + root_of(c, i), 1ull);
}

__global__ void k_keep_in_roots(CsfView c, const uint8_t *__restrict__ keep, int64_t a,
                                int64_t b, uint8_t *__restrict__ out) {
  const int64_t n = c.N[c.k - 1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t r = root_of(c, i);
    out[i] = (r >= a && r < b) ? keep[i] : (uint8_t)0;
  }
}

}  // namespace

int csf_root_counts(const CsfView &c, const uint8_t *d_keep, int64_t *d_cnt, cudaStream_t s) {
  VX_CUDA(cudaMemsetAsync(d_cnt, 0, sizeof(int64_t) * (size_t)std::max<int64_t>(c.N[0], 1), s));
  if (c.N[c.k - 1] == 0) return VX_OK;
  k_root_counts<<<blocks_for(c.N[c.k - 1]), 256, 0, s>>>(c, d_keep, (unsigned long long *)d_cnt);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

int csf_keep_in_roots(const CsfView &c, const uint8_t *d_keep, int64_t a, int64_t b,
                      uint8_t *d_out, cudaStream_t s) {
  if (c.N[c.k - 1] == 0) return VX_OK;
  k_keep_in_roots<<<blocks_for(c.N[c.k - 1]), 256, 0, s>>>(c, d_keep, a, b, d_out);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
}

int csf_prune_forest(const CsfView &in, const uint8_t *d_keep, int split, int32_t *d_index,
                     const int64_t *d_seg_off, int nseg, int64_t *d_seg_kept, cudaStream_t s,
                     CsfObj *out, Timer *tm, int64_t *h_seg_kept) {
  const int64_t cap = INT32_MAX;
  switch (in.k) {
    case 1: return prune_c<1>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
    case 2: return prune_c<2>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
    case 3: return prune_c<3>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
    case 4: return prune_c<4>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
    case 5: return prune_c<5>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
    default: return prune_c<6>(in, d_keep, split, d_index, s, out, tm, d_seg_off, nseg, d_seg_kept, cap, h_seg_kept);
  }
}

int csf_box_codes_dev(const CsfView &c, void *d_codes, cudaStream_t s) {
  if (c.N[c.k - 1] == 0) return VX_OK;
  if (c.k * c.level <= 32)
    k_box_codes<uint32_t><<<blocks_for(c.N[c.k - 1]), 256, 0, s>>>(c, (uint32_t *)d_codes);
  else
    k_box_codes<uint64_t><<<blocks_for(c.N[c.k - 1]), 256, 0, s>>>(c, (uint64_t *)d_codes);
  note_launch();
  VX_LAUNCH_CHECK();
  return VX_OK;
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
