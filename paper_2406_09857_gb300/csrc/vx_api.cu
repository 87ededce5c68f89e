// vx_api.cu -- host runtime and C ABI of libvx (declared in include/vx.h).
//
//   - packing of the polynomials for the device (Sec. 2.1, polynomial as a tree of exponent
//     tuples), re-laid out fibre-major per partial-evaluation stage;
//   - grid levels of a domain (Sec. 3.2: level l bisects the domain 2^l times per axis);
//   - the level loop of Algorithm 3 with criterion C0 (Sec. 3.2), optionally in binary32
//     midpoint-radius below the last level and with binary64 rechecks;
//   - CSF, system and result objects, errors and kernel timing.
#include <cuda_runtime.h>

#include <unistd.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "vx_internal.cuh"

namespace vx {

// ---------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------
static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

static std::atomic<int64_t> g_launches{0};
void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::atomic<int> g_sm_count[64];
int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  int n = g_sm_count[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
    g_sm_count[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

// ---------------------------------------------------------------------------------------
// device memory: stream-ordered allocations from the device's default pool, which keeps
// freed memory cached for the next level instead of returning it to the driver.
// ---------------------------------------------------------------------------------------
static bool g_pool_ready[64] = {false};

int dmalloc(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  VX_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !g_pool_ready[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    g_pool_ready[dev] = true;
  }
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(p, bytes, s);
  if (e != cudaSuccess) {
    set_error("cudaMallocAsync(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA;
  }
  return VX_OK;
}

void dfree(void *p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------------------------------
// kernel timing
// ---------------------------------------------------------------------------------------
static int take_event(std::vector<cudaEvent_t> &pool, cudaEvent_t *e) {
  if (!pool.empty()) {
    *e = pool.back();
    pool.pop_back();
    return VX_OK;
  }
  VX_CUDA(cudaEventCreate(e));
  return VX_OK;
}

int Timer::begin(int kind, int64_t w) {
  Pending p;
  p.kind = kind;
  p.work = w;
  VX_CHECK(take_event(pool, &p.a));
  VX_CHECK(take_event(pool, &p.b));
  VX_CUDA(cudaEventRecord(p.a, stream));
  pending.push_back(p);
  return VX_OK;
}

int Timer::end() {
  if (pending.empty()) return VX_OK;
  VX_CUDA(cudaEventRecord(pending.back().b, stream));
  return VX_OK;
}

int Timer::collect() {
  if (pending.empty()) return VX_OK;
  VX_CUDA(cudaEventSynchronize(pending.back().b));
  for (auto &p : pending) {
    float t = 0.f;
    VX_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
    ms[p.kind] += t;
    launches[p.kind] += 1;
    work[p.kind] += p.work;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pending.clear();
  return VX_OK;
}

void Timer::release() {
  for (auto &p : pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
  pending.clear();
  pool.clear();
}

static const char *kKindNames[KK_COUNT] = {
    "stage0_fp64",  "stagej_fp64",  "leaf_fp64", "stage0_midrad", "stagej_midrad",
    "leaf_midrad",  "stage0_fp32",  "stagej_fp32", "leaf_fp32",   "csf_build",
    "prune_scan",   "split",        "compact",     "recheck_select", "stage0_pair",
    "stagej_pair",  "leaf_pair"};

// ---------------------------------------------------------------------------------------
// grid levels: box t on axis i is [lo + t w, lo + (t+1) w], w = (hi - lo) / 2^level.
// Accepted only when every grid point is a binary64, so that endpoints are exact and child
// boxes are subsets of their parents (the subdivision then never loses a box that a finer
// level would keep).
// ---------------------------------------------------------------------------------------
static int low_bit_exponent(double x) {  // x = M 2^e with M odd: returns e (x != 0)
  int e = 0;
  double m = std::frexp(std::fabs(x), &e);
  uint64_t M = (uint64_t)std::ldexp(m, 53);
  int tz = 0;
  while (!(M & 1)) {
    M >>= 1;
    ++tz;
  }
  return e - 53 + tz;
}

static bool grid_exact(double lo, double step, int64_t count, int mant_bits, int min_exp) {
  // all lo + t*step, 0 <= t <= count, are integers times 2^q below 2^mant_bits
  int q = 1 << 20;
  if (lo != 0.0) q = std::min(q, low_bit_exponent(lo));
  q = std::min(q, low_bit_exponent(step));
  if (q < min_exp) return false;
  double L = std::ldexp(lo, -q), W = std::ldexp(step, -q);
  double lim = std::ldexp(1.0, mant_bits);
  if (std::fabs(L) >= lim || std::fabs(W) >= lim) return false;
  long double last = (long double)L + (long double)count * (long double)W;
  return std::fabs((double)last) < lim && (long double)(double)last == last;
}

static bool api_trace() {
  static int on = -1;
  if (on < 0) on = std::getenv("VX_TRACE") ? 1 : 0;
  return on == 1;
}

static int make_grid(int k, const double *dom, int level, LevelGrid *g) {
  if (api_trace()) std::fprintf(stderr, "[vx] make_grid k=%d level=%d\n", k, level);
  if (!dom) {
    set_error("domain is NULL");
    return VX_EINVAL;
  }
  if (level < 0 || level > VX_MAXLEVEL) {
    set_error("level %d outside [0, %d]", level, VX_MAXLEVEL);
    return VX_EINVAL;
  }
  *g = LevelGrid{};
  for (int i = 0; i < k; ++i) {
    const double lo = dom[2 * i], hi = dom[2 * i + 1];
    if (!std::isfinite(lo) || !std::isfinite(hi) || !(lo < hi)) {
      set_error("axis %d: domain [%g, %g] must be finite with lo < hi", i, lo, hi);
      return VX_EINVAL;
    }
    const double w = hi - lo;
    if (w - hi != -lo || !std::isfinite(w)) {  // hi - lo must be exact
      set_error("axis %d: hi - lo is not a binary64", i);
      return VX_EINVAL;
    }
    const double wl = std::ldexp(w, -level);
    const int64_t count = (int64_t)1 << level;
    if (std::ldexp(wl, level) != w || !grid_exact(lo, wl, count, 53, -1074)) {
      set_error("axis %d: the level-%d grid of [%.17g, %.17g] is not exactly representable "
                "(use a dyadic domain)", i, level, lo, hi);
      return VX_EINVAL;
    }
    AxisGrid &a = g->ax[i];
    a.lo = lo;
    a.w = wl;
    const double hw = 0.5 * wl;
    if (api_trace()) std::fprintf(stderr, "[vx] axis %d exact64 ok\n", i);
    a.fexact = grid_exact(lo, hw, 2 * count, 24, -149) ? 1 : 0;
    if (api_trace()) std::fprintf(stderr, "[vx] axis %d fexact=%d\n", i, a.fexact);
    a.flo = (float)lo;
    a.fw = (float)wl;
    if (a.fexact && ((double)a.flo != lo || (double)a.fw != wl)) a.fexact = 0;
  }
  return VX_OK;
}

// ---------------------------------------------------------------------------------------
// polynomial packing
// ---------------------------------------------------------------------------------------
// uint64 monomial key -> int32 index, open addressing with linear probing (the packing looks
// up every term once per stage; a node-based map made that the bulk of packing time).
class FlatMap {
 public:
  void reserve(size_t n) {
    size_t cap = 16;
    while (cap < 2 * n) cap <<= 1;
    keys_.assign(cap, 0);
    vals_.assign(cap, -1);
    mask_ = cap - 1;
  }
  void put(uint64_t key, int32_t v) {
    size_t i = slot(key);
    while (vals_[i] >= 0 && keys_[i] != key) i = (i + 1) & mask_;
    keys_[i] = key;
    vals_[i] = v;
  }
  int32_t get(uint64_t key) const {  // -1 if absent
    if (vals_.empty()) return -1;
    size_t i = slot(key);
    while (vals_[i] >= 0) {
      if (keys_[i] == key) return vals_[i];
      i = (i + 1) & mask_;
    }
    return -1;
  }

 private:
  size_t slot(uint64_t key) const {
    uint64_t z = key + 0x9e3779b97f4a7c15ull;  // SplitMix64's finaliser as the hash
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (size_t)(z ^ (z >> 31)) & mask_;
  }
  std::vector<uint64_t> keys_;
  std::vector<int32_t> vals_;
  size_t mask_ = 0;
};

// Monomials in m variables (fields of b bits in a key, most significant first) -> an index:
// a table over every exponent vector below R = E + 1 in each variable (mixed radix R) when
// R^m is small, the hash map otherwise.
class KeyIndex {
 public:
  void build(const std::vector<uint64_t> &keys, int m, int b, int32_t E) {
    m_ = m;
    b_ = b;
    R_ = (int64_t)E + 1;
    int64_t size = 1;
    dense_ = true;
    for (int j = 0; j < m && dense_; ++j) {
      size *= R_;
      dense_ = size <= ((int64_t)1 << 22);
    }
    if (dense_) {
      tab_.assign((size_t)size, -1);
      for (size_t f = 0; f < keys.size(); ++f) {
        const int64_t ix = of_key(keys[f]);
        if (ix >= 0) tab_[(size_t)ix] = (int32_t)f;
      }
    } else {
      map_.reserve(keys.size());
      for (size_t f = 0; f < keys.size(); ++f) map_.put(keys[f], (int32_t)f);
    }
  }
  int32_t get_key(uint64_t key) const {  // -1 if absent
    if (!dense_) return map_.get(key);
    const int64_t ix = of_key(key);
    return ix < 0 ? -1 : tab_[(size_t)ix];
  }
  // the monomial of exponents e[from..k-1] (m = k - from of them)
  int32_t get(const int32_t *e, int from, int k) const {
    if (!dense_) {
      uint64_t key = 0;
      for (int v = from; v < k; ++v) key = (key << b_) | (uint64_t)e[v];
      return map_.get(key);
    }
    int64_t ix = 0;
    for (int v = from; v < k; ++v) {
      if (e[v] >= R_) return -1;
      ix = ix * R_ + e[v];
    }
    return tab_[(size_t)ix];
  }

 private:
  int64_t of_key(uint64_t key) const {
    const uint64_t mask = b_ >= 64 ? ~0ull : ((1ull << b_) - 1);
    int64_t ix = 0;
    for (int j = 0; j < m_; ++j) {
      const int64_t e = (int64_t)((key >> (b_ * (m_ - 1 - j))) & mask);
      if (e >= R_) return -1;
      ix = ix * R_ + e;
    }
    return ix;
  }
  bool dense_ = false;
  int m_ = 0, b_ = 0;
  int64_t R_ = 0;
  std::vector<int32_t> tab_;
  FlatMap map_;
};

struct HostStage {
  int32_t nfib = 0, maxlen = 0;
  int64_t blk_in = 0, blk_out = 0;
  std::vector<uint64_t> keys;  // fibre monomial in x_{s+2}..x_k, key_bits(k) bits per exponent
  std::vector<int32_t> rowoff, fiblen, outpos, fiboff, outpos_fm;
  KeyIndex index;
};

struct HostPoly {
  HostStage st[VX_KMAX];  // the coefficient block (st[0].blk_in entries) is packed by pack_coefs
};

// A monomial in up to k - 1 variables packed into 64 bits: 16 bits per exponent up to
// k = 5, 64 / (k - 1) bits beyond (12 bits at k = 6).
static int key_bits(int k) { return k <= 5 ? 16 : 64 / (k - 1); }

// The binary32 encodings of the stage-0 coefficient block, made on the device from the
// binary64 intervals [c.x, c.y] (c.x = c.y for a point coefficient):
//  - midpoint-radius <m, r>: m = RN of the midpoint, r >= the larger distance to an end plus
//    2^-149 (which pays for the rounding of the Horner step that adds this coefficient when
//    its result falls below the normal range);
//  - certified (RN(lo), -RN(hi)) and a bound E >= (1 + 2^-39)(d + 2^-24 max(|lo|, |hi|)) +
//    2^-148, d the larger distance of the two ends to their binary64 values (which the
//    binary64 path uses as they are); the 2^-24 term keeps E >= 2^-24 max(|RN(lo)|,
//    |RN(hi)|), which the error recursion of the evaluation kernels relies on.  E is stored
//    twice (.z and .w): a register pair for the kernels' paired steps.
//  - float pairs (eval_level_pair): each end c as h = RN(c), l = RN(c - h) (c - (h + l) is
//    exact in binary64), stored (lo_h, lo_l, -hi_h, -hi_l), with the bound RU(max of the two
//    representation errors) + 2^-148; a non-finite pair gets an infinite bound.
__global__ void k_encode_coefs(const double2 *__restrict__ c64, int64_t n, float2 *__restrict__ c32,
                               float4 *__restrict__ c32c, float4 *__restrict__ cp,
                               float *__restrict__ ep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double lo = c64[i].x, hi = c64[i].y;
    {
      const float lh = __double2float_rn(lo), hh = __double2float_rn(hi);
      const float ll = __double2float_rn(lo - (double)lh), hl = __double2float_rn(hi - (double)hh);
      const double d = fmax(fabs((lo - (double)lh) - (double)ll), fabs((hi - (double)hh) - (double)hl));
      cp[i] = make_float4(lh, ll, -hh, -hl);
      ep[i] = (isfinite(lh) && isfinite(hh) && isfinite(ll) && isfinite(hl))
                  ? __double2float_ru(__dadd_ru(d, 0x1p-148))
                  : INFINITY;
    }
    {
      const double mid = lo == hi ? lo : __dadd_rn(__dmul_rn(0.5, lo), __dmul_rn(0.5, hi));
      const float m = __double2float_rn(mid);
      if (!isfinite(m)) {
        c32[i] = make_float2(0.f, INFINITY);
      } else {
        const double dm = (double)m;
        // |end - m| for the farther end, rounded up, padded for the ulp of the midpoint
        const double d = fmax(__dadd_ru(hi, -dm), __dadd_ru(dm, -lo));
        c32[i] = make_float2(m, __double2float_ru(__dadd_ru(__dmul_ru(d, 1.0 + 0x1p-50), 0x1p-149)));
      }
    }
    {
      const float flo = __double2float_rn(lo), fhi = __double2float_rn(hi);
      if (!isfinite(flo) || !isfinite(fhi)) {
        c32c[i] = make_float4(-INFINITY, -INFINITY, INFINITY, INFINITY);
      } else {
        const double d = fmax(fabs(lo - (double)flo), fabs(hi - (double)fhi));  // exact
        const double mag = fmax(fabs(lo), fabs(hi));
        // (mag 2^-24 may round below the double range; the 2^-148 term covers it)
        const double bound = __dmul_ru(__dadd_ru(d, __dmul_ru(mag, 0x1p-24)), 1.0 + 0x1p-39);
        const float e = __double2float_ru(__dadd_ru(bound, 0x1p-148));
        c32c[i] = make_float4(flo, -fhi, e, e);
      }
    }
  }
}

// The stage-0 blocks fibre-major: entry a of fibre f (row-major at rowoff[a] + f) to
// fiboff[f] + a, so that a stage-0 Horner walks consecutive entries; every encoding of the
// coefficients (binary64 intervals, midpoint-radius, certified binary32, float pairs and their
// bounds) is permuted the same way.
struct Stage0Blocks {
  const double2 *c64;
  const float2 *c32;
  const float4 *c32c, *cp;
  const float *ep;
};
struct Stage0BlocksFm {
  double2 *c64;
  float2 *c32;
  float4 *c32c, *cp;
  float *ep;
};
// A warp per fibre, its lanes over the fibre's entries (writes coalesced).
__global__ void k_fibre_major(Stage0Blocks r, const int32_t *__restrict__ rowoff,
                              const int32_t *__restrict__ fiblen,
                              const int32_t *__restrict__ fiboff, int32_t nfib,
                              Stage0BlocksFm w) {
  const int wpb = (int)(blockDim.x >> 5), lane = (int)(threadIdx.x & 31);
  const int stride = (int)gridDim.x * wpb;
  for (int f = (int)blockIdx.x * wpb + (int)(threadIdx.x >> 5); f < nfib; f += stride) {
    const int L = fiblen[f], o = fiboff[f];
    for (int a = lane; a < L; a += 32) {
      const int i = rowoff[a] + f;
      w.c64[o + a] = r.c64[i];
      w.c32[o + a] = r.c32[i];
      w.c32c[o + a] = r.c32c[i];
      w.cp[o + a] = r.cp[i];
      w.ep[o + a] = r.ep[i];
    }
  }
}

// chi (nullable): upper ends of interval coefficients [p.coefs[t], chi[t]]
// Host threads kept for the process (one per core but this one's, at most 15): run(n, fn)
// calls fn(c) for c = 0..n-1 on them and on the calling thread and returns when all are done.
// One job at a time: a caller that finds the pool busy gets false and nothing runs.
class HostPool {
 public:
  static HostPool &get() {
    // never destroyed (its threads live as long as the process); a process forked from this
    // one has none of its threads and maybe a lock taken at the fork, so it makes its own
    static std::mutex mu;
    static HostPool *p = nullptr;
    static pid_t owner = 0;
    std::lock_guard<std::mutex> g(mu);
    if (!p || owner != getpid()) {
      p = new HostPool();
      owner = getpid();
    }
    return *p;
  }
  int size() const { return (int)nworkers_ + 1; }
  template <class Fn>
  bool run(int n, Fn &&fn) {
    std::unique_lock<std::mutex> busy(busy_, std::try_to_lock);
    if (!busy.owns_lock()) return false;
    std::function<void(int)> f(fn);
    {
      std::lock_guard<std::mutex> g(m_);
      job_ = &f;
      n_ = n;
      next_.store(0);
      ++gen_;
      gen_pub_.store(gen_, std::memory_order_release);
    }
    cv_.notify_all();
    drain();
    // the workers' last chunks usually end within microseconds: wait for them spinning first
    spin_until([&] { return active_.load(std::memory_order_acquire) == 0; });
    std::unique_lock<std::mutex> g(m_);
    done_.wait(g, [&] { return active_.load() == 0; });  // every chunk a worker took has finished
    job_ = nullptr;
    return true;
  }

 private:
  HostPool() {
    const int hw = (int)std::thread::hardware_concurrency();
    nworkers_ = std::max(0, std::min(15, hw - 1));
    for (int i = 0; i < nworkers_; ++i) std::thread([this] { loop(); }).detach();
  }
  void drain() {
    for (;;) {
      const int c = next_.fetch_add(1);
      if (c >= n_) return;
      (*job_)(c);
    }
  }
  // Spins until pred() holds or kSpinUs microseconds pass: packing issues its jobs back to
  // back, and a wake-up through a condition variable costs tens of microseconds each.
  static constexpr int kSpinUs = 200;
  template <class Pred>
  static void spin_until(Pred pred) {
    const auto t0 = std::chrono::steady_clock::now();
    while (!pred() && std::chrono::steady_clock::now() - t0 < std::chrono::microseconds(kSpinUs)) {
    }
  }
  void loop() {
    uint64_t seen = 0;
    for (;;) {
      spin_until([&] { return gen_pub_.load(std::memory_order_acquire) != seen; });
      std::unique_lock<std::mutex> g(m_);
      cv_.wait(g, [&] { return gen_ != seen && job_ != nullptr; });
      seen = gen_;
      active_.fetch_add(1);
      g.unlock();
      drain();
      g.lock();
      if (active_.fetch_sub(1) == 1) done_.notify_all();
    }
  }
  int nworkers_ = 0;
  std::mutex busy_, m_;
  std::condition_variable cv_, done_;
  std::function<void(int)> *job_ = nullptr;
  int n_ = 0;
  std::atomic<int> active_{0};  // changed under m_; read without it while spinning
  uint64_t gen_ = 0;
  std::atomic<uint64_t> gen_pub_{0};  // gen_, for the workers' spin
  std::atomic<int> next_{0};
};

// Polynomials with at least this many terms split their packing loops over the host pool
// (smaller ones, e.g. a batch's, are packed by many callers at once already).
constexpr int32_t kPackSplitTerms = 50000;

// fn(c, begin, end) on chunk c of nchunks contiguous chunks of [0, n), on the host pool when
// there are several chunks and it is free, else on this thread.
template <class Fn>
static void for_chunks(int64_t n, int nchunks, Fn fn) {
  const int64_t per = (n + nchunks - 1) / std::max(nchunks, 1);
  auto chunk = [&](int c) {
    const int64_t a = c * per, b = std::min<int64_t>(n, a + per);
    if (a < b) fn(c, a, b);
  };
  if (nchunks > 1 && HostPool::get().run(nchunks, chunk)) return;
  for (int c = 0; c < nchunks; ++c) chunk(c);
}

// The checks and the layout of a polynomial (each stage's fibres, offsets and output
// positions); its coefficient block comes from pack_coefs.  chunks: pieces of the loops over
// the terms (several for large polynomials: host pool).
static int pack_poly(int k, const vx_poly &p, HostPoly *hp, const double *chi = nullptr,
                     int chunks = 1) {
  const int32_t nt = p.nterms;
  if (p.nvars != k || nt < 0 || (nt > 0 && (!p.exps || !p.coefs))) {
    set_error("polynomial: nvars %d (expected %d), nterms %d", p.nvars, k, nt);
    return VX_EINVAL;
  }
  const int T = std::max(1, std::min(chunks, 64));
  const int32_t emax = (1 << key_bits(k)) - 1;
  int32_t E = 0;  // the largest exponent of any variable
  {
    // the first bad exponent and the first bad coefficient (each chunk its own first)
    std::vector<int64_t> bad_e(T, -1), bad_c(T, -1);
    std::vector<int32_t> top(T, 0);
    for_chunks(nt, T, [&](int c, int64_t a, int64_t b) {
      int32_t mx = 0;
      for (int64_t t = a * k; t < b * k; ++t) {
        if (p.exps[t] < 0 || p.exps[t] > emax) {
          bad_e[c] = t;
          break;
        }
        mx = std::max(mx, p.exps[t]);
      }
      top[c] = mx;
      for (int64_t t = a; t < b; ++t)
        if (!std::isfinite(p.coefs[t]) ||
            (chi && !(std::isfinite(chi[t]) && chi[t] >= p.coefs[t]))) {
          bad_c[c] = t;
          break;
        }
    });
    for (int c = 0; c < T; ++c)
      if (bad_e[c] >= 0) {
        set_error("polynomial: exponent %d outside [0, %d]", p.exps[bad_e[c]], emax);
        return VX_EINVAL;
      }
    for (int c = 0; c < T; ++c) E = std::max(E, top[c]);
    for (int c = 0; c < T; ++c)
      if (bad_c[c] >= 0) {
        set_error("polynomial: coefficient %d is not finite (or not an interval)", (int)bad_c[c]);
        return VX_EINVAL;
      }
  }
  // closure of the fibre sets, last stage first: stage s's fibres are the entries of stage
  // s+1's input (monomials in x_{s+2}..x_k), each as long as the highest exponent of
  // x_{s+1} among the terms with that monomial (1 if none: an all-zero fibre)
  hp->st[k - 1].keys.assign(1, 0);
  for (int s = k - 1; s >= 0; --s) {
    HostStage &S = hp->st[s];
    const int32_t nf = (int32_t)S.keys.size();
    KeyIndex idx;
    idx.build(S.keys, k - 1 - s, key_bits(k), E);
    // per chunk of terms the longest fibre lengths, then their maxima
    std::vector<std::vector<int32_t>> lens(T);
    std::vector<uint8_t> miss(T, 0);
    for_chunks(nt, T, [&](int c, int64_t a, int64_t b) {
      std::vector<int32_t> &len = lens[c];
      len.assign(nf, 1);
      for (int64_t t = a; t < b; ++t) {
        const int32_t *e = p.exps + t * k;
        const int32_t g = idx.get(e, s + 1, k);
        if (g < 0) {
          miss[c] = 1;
          return;
        }
        len[g] = std::max(len[g], e[s] + 1);
      }
    });
    for (int c = 0; c < T; ++c)
      if (miss[c]) {
        set_error("internal: monomial outside the fibre closure");
        return VX_EINVAL;
      }
    std::vector<int32_t> len(nf, 1);
    for (int c = 0; c < T; ++c)
      if (!lens[c].empty())
        for (int32_t f = 0; f < nf; ++f) len[f] = std::max(len[f], lens[c][f]);
    // the fibres longest first, equal lengths by increasing key: a counting sort by length,
    // then each length's keys sorted
    int32_t maxl = 1;
    for (int32_t f = 0; f < nf; ++f) maxl = std::max(maxl, len[f]);
    std::vector<int32_t> start(maxl + 2, 0);  // bucket b = maxl - length
    for (int32_t f = 0; f < nf; ++f) ++start[maxl - len[f] + 1];
    for (int32_t b = 0; b <= maxl; ++b) start[b + 1] += start[b];
    std::vector<uint64_t> keys(nf);
    {
      std::vector<int32_t> next(start.begin(), start.end() - 1);
      for (int32_t f = 0; f < nf; ++f) keys[next[maxl - len[f]]++] = S.keys[f];
    }
    S.fiblen.resize(nf);
    for (int32_t b = 0; b <= maxl; ++b) {
      std::sort(keys.begin() + start[b], keys.begin() + start[b + 1]);
      for (int32_t f = start[b]; f < start[b + 1]; ++f) S.fiblen[f] = maxl - b;
    }
    S.keys.swap(keys);
    S.index.build(S.keys, k - 1 - s, key_bits(k), E);
    S.nfib = nf;
    S.maxlen = S.fiblen[0];
    S.rowoff.assign(S.maxlen + 1, 0);
    {
      int32_t f = nf;  // fibres with len > a form the prefix 0..cnt(a)-1
      for (int32_t a = 0; a < S.maxlen; ++a) {
        while (f > 0 && S.fiblen[f - 1] <= a) --f;
        S.rowoff[a + 1] = S.rowoff[a] + f;
      }
    }
    S.blk_in = S.rowoff[S.maxlen];
    S.fiboff.assign(nf + 1, 0);
    for (int32_t f = 0; f < nf; ++f) S.fiboff[f + 1] = S.fiboff[f] + S.fiblen[f];
    if (S.maxlen > 8192) {
      set_error("polynomial: degree %d in one variable exceeds 8191", S.maxlen - 1);
      return VX_EINVAL;
    }
    if (S.blk_in > INT32_MAX / 2) {
      set_error("polynomial too large: %lld coefficients in one stage", (long long)S.blk_in);
      return VX_EINVAL;
    }
    if (s > 0) {
      std::vector<uint64_t> &nk = hp->st[s - 1].keys;
      nk.clear();
      nk.reserve(S.blk_in);
      const int sh = key_bits(k) * (k - 1 - s);
      for (int32_t f = 0; f < nf; ++f)
        for (int32_t a = 0; a < S.fiblen[f]; ++a) nk.push_back(((uint64_t)a << sh) | S.keys[f]);
    }
  }
  for (int s = 0; s < k; ++s) {
    HostStage &S = hp->st[s];
    S.blk_out = s + 1 < k ? hp->st[s + 1].blk_in : 1;
    S.outpos.assign(S.nfib, 0);
    S.outpos_fm.assign(S.nfib, 0);
    if (s + 1 < k) {
      const HostStage &T = hp->st[s + 1];
      const int sh = key_bits(k) * (k - 2 - s);
      const uint64_t mask = sh ? ((uint64_t)1 << sh) - 1 : 0;
      for (int32_t f = 0; f < S.nfib; ++f) {
        const uint64_t a = S.keys[f] >> sh;
        const int32_t g = T.index.get_key(S.keys[f] & mask);
        S.outpos[f] = T.rowoff[a] + g;
        S.outpos_fm[f] = T.fiboff[g] + (int32_t)a;
      }
    }
  }
  return VX_OK;
}

// The coefficient block of stage 0 (entry (a_1, fibre) at rowoff[a_1] + fibre) of a packed
// polynomial, written to dst (st[0].blk_in entries: the staging buffer of the upload, so that
// the block is neither built elsewhere first nor copied); entries of no term are zero.
static int pack_coefs(int k, const vx_poly &p, const HostPoly &hp, const double *chi,
                      double2 *dst, int chunks = 1) {
  const int32_t nt = p.nterms;
  const int T = std::max(1, std::min(chunks, 64));
  const HostStage &S0 = hp.st[0];
  const int64_t n = S0.blk_in;
  std::vector<uint8_t> seen((size_t)n);
  for_chunks(n, T, [&](int, int64_t a, int64_t b) {
    std::memset(dst + a, 0, (size_t)(b - a) * sizeof(double2));
    std::memset(seen.data() + a, 0, (size_t)(b - a));
  });
  std::vector<int64_t> dup(T, -1);
  for_chunks(nt, T, [&](int c, int64_t a, int64_t b) {
    for (int64_t t = a; t < b; ++t) {
      const int32_t *e = p.exps + t * k;
      const int32_t f = S0.index.get(e, 1, k);
      const int64_t pos = S0.rowoff[e[0]] + f;
      // a monomial seen before, by this chunk or another one (atomic: chunks run at once)
      if (__atomic_exchange_n(&seen[pos], (uint8_t)1, __ATOMIC_RELAXED)) {
        if (dup[c] < 0) dup[c] = t;
        continue;
      }
      dst[pos] = make_double2(p.coefs[t], chi ? chi[t] : p.coefs[t]);
    }
  });
  for (int c = 0; c < T; ++c)
    if (dup[c] >= 0) {
      set_error("polynomial: monomial %d appears twice", (int)dup[c]);
      return VX_EINVAL;
    }
  return VX_OK;
}

}  // namespace vx

namespace vx {

// One level in one mode.  The binary32 modes flag boxes for a binary64 re-evaluation (VX_FP32:
// those inside the error band; VX_FP32_MIDRAD with recheck: the tight ones); flagged boxes are
// gathered into a tree of their own, evaluated in binary64 and their decisions scattered back.
// defer (VX_FP32): no re-evaluation, the band's boxes are kept.
// Certified binary32 levels whose band is re-decided now go through the float-pair tier.
static bool flagged_pair_tier(int mode, bool defer) { return mode == VX_FP32 && !defer; }

// The boxes of tree c whose flag is set, as a tree of their own (their tuples are increasing,
// being listed in leaf order), decided in binary64; the decisions go to keep at their places.
static int decide_flagged_fp64(const SysDev &sys, const CsfView &c, const LevelGrid &g,
                               const uint8_t *flag, uint8_t *keep, cudaStream_t s, Timer *tm,
                               int64_t *madds, int64_t *nsel) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  int32_t *idx = nullptr, *tup = nullptr;
  uint8_t *subkeep = nullptr;
  int64_t ns = 0;
  *nsel = 0;
  int rc = VX_OK;
  if (tm && tm->on) rc = tm->begin(KK_RECHECK, n);
  if (rc == VX_OK) rc = flag_indices(flag, n, s, &idx, &ns);
  if (rc == VX_OK && tm && tm->on) {
    tm->add_work(4 * ns);  // the selected boxes' indices written
    rc = tm->end();
  }
  *nsel = ns;
  if (rc == VX_OK && ns > 0) {
    CsfObj sub;
    rc = dmalloc((void **)&tup, (size_t)ns * k * 4, s);
    if (rc == VX_OK) rc = csf_tuples_of(c, idx, ns, tup, s);
    if (rc == VX_OK) rc = csf_build_dev(k, c.level, tup, ns, s, &sub, tm);
    if (rc == VX_OK) rc = dmalloc((void **)&subkeep, (size_t)ns, s);
    int64_t w2 = 0;
    if (rc == VX_OK)
      rc = eval_level_raw(sys, sub.v, g, ARITH_F64, nullptr, nullptr, subkeep, nullptr, 0.f, s,
                          tm, &w2);
    *madds += w2;
    if (rc == VX_OK) rc = scatter_keep(idx, subkeep, ns, keep, s);
    csf_release(&sub);
  }
  dfree(subkeep, s);
  dfree(tup, s);
  dfree(idx, s);
  return rc;
}

static int eval_decide(const SysDev &sys, const CsfView &c, const LevelGrid &g, int mode,
                       bool midrad_recheck, float theta, double *d_lo, double *d_hi,
                       uint8_t *keep, cudaStream_t s, Timer *tm, int64_t *madds,
                       int64_t *nrecheck, bool defer = false, int64_t *nrecheck64 = nullptr) {
  const int k = c.k;
  const int64_t n = c.N[k - 1];
  *madds = 0;
  *nrecheck = 0;
  if (nrecheck64) *nrecheck64 = 0;
  if (flagged_pair_tier(mode, defer) && n > 0) {
    // certified binary32, then the float-pair tier on its error band, then binary64 on what
    // the tier leaves undecided
    uint8_t *flag = nullptr;
    VX_CHECK(dmalloc((void **)&flag, (size_t)n, s));
    int rc = eval_level_raw(sys, c, g, ARITH_F32_CERT, d_lo, d_hi, keep, flag, theta, s, tm, madds);
    int32_t *idx = nullptr, *tup = nullptr;
    uint8_t *subkeep = nullptr, *subflag = nullptr;
    int64_t ns = 0;
    if (rc == VX_OK && tm && tm->on) rc = tm->begin(KK_RECHECK, n);
    if (rc == VX_OK) rc = flag_indices(flag, n, s, &idx, &ns);
    if (rc == VX_OK && tm && tm->on) {
      tm->add_work(4 * ns);
      rc = tm->end();
    }
    *nrecheck = ns;
    if (rc == VX_OK && ns > 0) {
      CsfObj sub;
      rc = dmalloc((void **)&tup, (size_t)ns * k * 4, s);
      if (rc == VX_OK) rc = csf_tuples_of(c, idx, ns, tup, s);
      if (rc == VX_OK) rc = csf_build_dev(k, c.level, tup, ns, s, &sub, tm);
      if (rc == VX_OK) rc = dmalloc((void **)&subkeep, (size_t)ns, s);
      if (rc == VX_OK) rc = dmalloc((void **)&subflag, (size_t)ns, s);
      int64_t wp = 0, w64 = 0, n64 = 0;
      if (rc == VX_OK) rc = eval_level_pair(sys, sub.v, g, subkeep, subflag, s, tm, &wp);
      if (rc == VX_OK) rc = decide_flagged_fp64(sys, sub.v, g, subflag, subkeep, s, tm, &w64, &n64);
      *madds += wp + w64;
      if (nrecheck64) *nrecheck64 = n64;
      if (rc == VX_OK) rc = scatter_keep(idx, subkeep, ns, keep, s);
      csf_release(&sub);
    }
    dfree(subflag, s);
    dfree(subkeep, s);
    dfree(tup, s);
    dfree(idx, s);
    dfree(flag, s);
    return rc;
  }
  const bool flagged =
      (mode == VX_FP32 && !defer) || (mode == VX_FP32_MIDRAD && midrad_recheck);
  const int arith = mode == VX_FP64 ? ARITH_F64 : (mode == VX_FP32 ? ARITH_F32_CERT : ARITH_F32_MIDRAD);
  uint8_t *flag = nullptr;
  if (flagged) VX_CHECK(dmalloc((void **)&flag, (size_t)std::max<int64_t>(n, 1), s));
  int rc = eval_level_raw(sys, c, g, arith, d_lo, d_hi, keep, flag, theta, s, tm, madds);
  if (rc == VX_OK && flagged && n > 0) {
    // the flagged leaves as a tree of their own (their tuples are increasing, being listed in
    // leaf order), evaluated in binary64; the decisions go back to their places
    int32_t *idx = nullptr, *tup = nullptr;
    uint8_t *subkeep = nullptr;
    int64_t ns = 0;
    if (tm && tm->on) rc = tm->begin(KK_RECHECK, n);
    if (rc == VX_OK) rc = flag_indices(flag, n, s, &idx, &ns);
    if (rc == VX_OK && tm && tm->on) {
      tm->add_work(4 * ns);  // the selected boxes' indices written
      rc = tm->end();
    }
    *nrecheck = ns;
    if (rc == VX_OK && ns > 0) {
      CsfObj sub;
      rc = dmalloc((void **)&tup, (size_t)ns * k * 4, s);
      if (rc == VX_OK) rc = csf_tuples_of(c, idx, ns, tup, s);
      if (rc == VX_OK) rc = csf_build_dev(k, c.level, tup, ns, s, &sub, tm);
      if (rc == VX_OK) rc = dmalloc((void **)&subkeep, (size_t)ns, s);
      int64_t w2 = 0;
      if (rc == VX_OK)
        rc = eval_level_raw(sys, sub.v, g, ARITH_F64, nullptr, nullptr, subkeep, nullptr, 0.f, s,
                            tm, &w2);
      *madds += w2;
      if (rc == VX_OK) rc = scatter_keep(idx, subkeep, ns, keep, s);
      csf_release(&sub);
    }
    dfree(subkeep, s);
    dfree(tup, s);
    dfree(idx, s);
  }
  dfree(flag, s);
  return rc;
}

}  // namespace vx

using namespace vx;

struct vx_system {
  SysDev dev;
  void *mem = nullptr;
  size_t bytes = 0;
  size_t upload_bytes = 0;  // of them, copied from the host (the rest is made on the device)
  cudaStream_t stream = nullptr;
  std::vector<int64_t> M;  // [npoly][k+1]
  // the polynomials as given (exponents [nterms][k], coefficients), for dense-level plans
  std::vector<std::vector<int32_t>> exps;
  std::vector<std::vector<double>> coefs;
  std::vector<std::vector<double>> coefs_hi;  // upper ends of interval coefficients (or empty)
  // Taylor forms (Def. 3): per order m, per polynomial, the system of its G_a, made on first use
  struct TaylorSet {
    vx_system *sys = nullptr;
    std::vector<std::array<int8_t, VX_KMAX>> alpha;
  };
  std::mutex tmu;
  std::map<int, std::vector<TaylorSet>> taylor;
};

struct vx_csf {
  CsfObj o;
};

struct vx_result {
  int k = 0, depth = 0;
  // the final boxes: one tree, or (an enclosure run in x_1 ranges) fin and then the trees in
  // `more`, one after another in lexicographic order; `merged` joins them on request
  CsfObj fin;
  bool fin_set = false;
  std::vector<CsfObj> more;
  CsfObj merged;
  bool merged_set = false;
  std::vector<int64_t> tested, kept, nodes, recheck, madds;
  std::vector<int64_t> recheck64;  // of the rechecked boxes, those decided in binary64
  Timer tm;
  double elapsed_ms = 0.0;
  // the boxes on the host: a pinned buffer from the library's pool (vx_result_boxes)
  int32_t *htup = nullptr;
  size_t hcap = 0;       // bytes of the buffer
  int64_t hcount = -1;   // boxes copied (-1: not yet)
  // the boxes as grid indices on the host (vx_result_box_codes), a pinned pool buffer
  void *hcodes = nullptr;
  size_t hcodes_cap = 0;
  int64_t hcodes_count = -1;
  // with C1: the certified boxes of each level (device CSFs), and their host copy
  std::vector<std::pair<int, CsfObj>> incl;
  std::vector<int32_t> hinc_lev, hinc_tup;
  int64_t hinc_count = -1;
};

// ---------------------------------------------------------------------------------------
// Pinned host buffers for results' boxes, kept for reuse: device-to-host copies into pinned
// memory run at the link's rate (pageable copies go through a staging buffer), and pinning
// is paid once per buffer, not once per result.
// ---------------------------------------------------------------------------------------
// every device tree a result holds
static void result_release_trees(vx_result *R) {
  csf_release(&R->fin);
  for (auto &c : R->more) csf_release(&c);
  R->more.clear();
  if (R->merged_set) csf_release(&R->merged);
  R->merged_set = false;
  for (auto &lc : R->incl) csf_release(&lc.second);
  R->incl.clear();
}

// the final trees in order (fin first)
static std::vector<const CsfObj *> result_trees(const vx_result *R) {
  std::vector<const CsfObj *> t;
  t.push_back(&R->fin);
  for (auto &c : R->more) t.push_back(&c);
  return t;
}

static std::mutex g_pin_mu;
static std::multimap<size_t, void *> g_pin_free;  // capacity -> buffer

static int pinned_get(size_t bytes, void **p, size_t *cap) {
  {
    std::lock_guard<std::mutex> g(g_pin_mu);
    auto it = g_pin_free.lower_bound(bytes);
    if (it != g_pin_free.end() && it->first <= 2 * bytes + (64u << 20)) {
      *p = it->second;
      *cap = it->first;
      g_pin_free.erase(it);
      return VX_OK;
    }
  }
  const size_t c = (bytes + (16u << 20) - 1) & ~(size_t)((16u << 20) - 1);  // 16 MiB steps
  // mapped: the device can also write into it directly (the result's box codes)
  if (cudaHostAlloc(p, c, cudaHostAllocMapped) != cudaSuccess) {
    set_error("cudaHostAlloc of %zu bytes failed", c);
    return VX_ENOMEM;
  }
  *cap = c;
  return VX_OK;
}

// the box codes written by the device into the result's pinned buffer (else via device memory)
constexpr bool kCodesToHost = true;

static void pinned_put(void *p, size_t cap) {
  if (!p) return;
  std::lock_guard<std::mutex> g(g_pin_mu);
  g_pin_free.emplace(cap, p);
  // keep the pool bounded: release the largest buffers beyond 8
  while (g_pin_free.size() > 8) {
    auto it = std::prev(g_pin_free.end());
    cudaFreeHost(it->second);
    g_pin_free.erase(it);
  }
}

static cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------
extern "C" {

const char *vx_last_error(void) { return g_err; }

// keep_host: keep a host copy of the polynomials (the dense plan and the Taylor form's derived
// system are made from it later); a system that one call creates, uses and frees need not
static int system_create_impl(const vx_poly *F, int32_t npoly, const double *const *chi,
                              void *stream, vx_system **out, const int32_t *rel = nullptr,
                              bool keep_host = true);

int vx_system_create(const vx_poly *F, int32_t npoly, void *stream, vx_system **out) {
  clear_error();
  return system_create_impl(F, npoly, nullptr, stream, out);
}

int vx_system_create_ex(const vx_poly *F, const double *const *coefs_hi, const int32_t *rel,
                        int32_t npoly, void *stream, vx_system **out) {
  clear_error();
  return system_create_impl(F, npoly, coefs_hi, stream, out, rel);
}

// chi (nullable; entries nullable): per polynomial, the upper ends of interval coefficients
// (F[f].coefs the lower ends); rel (nullable): the relation of each polynomial.
static int system_create_impl(const vx_poly *F, int32_t npoly, const double *const *chi,
                              void *stream, vx_system **out, const int32_t *rel, bool keep_host) {
  if (!out || !F || npoly < 1 || npoly > VX_MAXPOLY) {
    set_error("vx_system_create: need 1..%d polynomials and an out pointer", VX_MAXPOLY);
    return VX_EINVAL;
  }
  for (int f = 0; rel && f < npoly; ++f)
    if (rel[f] < VX_EQ || rel[f] > VX_GT) {
      set_error("vx_system_create: polynomial %d has an unknown relation %d", f, rel[f]);
      return VX_EINVAL;
    }
  *out = nullptr;
  const int k = F[0].nvars;
  if (k < 1 || k > VX_KMAX) {
    set_error("vx_system_create: %d variables (1..%d supported)", k, VX_KMAX);
    return VX_EINVAL;
  }
  std::vector<HostPoly> hp(npoly);
  int64_t terms = 0;
  for (int f = 0; f < npoly; ++f) terms += std::max<int32_t>(F[f].nterms, 0);
  const int pool_chunks = 2 * HostPool::get().size();
  bool large = false;
  for (int f = 0; f < npoly; ++f) large = large || F[f].nterms >= kPackSplitTerms;
  if (large) {
    // large polynomials one after another, each one's loops over its terms on the host pool
    for (int f = 0; f < npoly; ++f)
      VX_CHECK(pack_poly(k, F[f], &hp[f], chi ? chi[f] : nullptr,
                         F[f].nterms >= kPackSplitTerms ? pool_chunks : 1));
  } else if (npoly > 1 && terms >= 20000) {
    // mid-sized polynomials pack concurrently (host work, one thread each)
    std::vector<int> rcs(npoly, VX_OK);
    std::vector<std::string> msgs(npoly);
    std::vector<std::thread> th;
    for (int f = 0; f < npoly; ++f)
      th.emplace_back([&, f] {
        rcs[f] = pack_poly(k, F[f], &hp[f], chi ? chi[f] : nullptr);
        if (rcs[f] != VX_OK) msgs[f] = vx_last_error();
      });
    for (auto &t : th) t.join();
    for (int f = 0; f < npoly; ++f)
      if (rcs[f] != VX_OK) {
        set_error("%s", msgs[f].c_str());
        return rcs[f];
      }
  } else {
    for (int f = 0; f < npoly; ++f) VX_CHECK(pack_poly(k, F[f], &hp[f], chi ? chi[f] : nullptr));
  }
  // one device allocation: per polynomial the coefficient blocks, then per stage the row
  // offsets, fibre lengths, output positions, fibre-major offsets and output positions
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t bytes = 0;
  for (int f = 0; f < npoly; ++f) {
    const size_t nc = (size_t)hp[f].st[0].blk_in;
    bytes += 2 * al(nc * sizeof(double2)) + 2 * al(nc * sizeof(float2)) + 4 * al(nc * sizeof(float4)) +
             2 * al(nc * sizeof(float));
    for (int s = 0; s < k; ++s) {
      const HostStage &S = hp[f].st[s];
      bytes += al((S.maxlen + 1) * 4) + 3 * al((size_t)S.nfib * 4) + al(((size_t)S.nfib + 1) * 4);
    }
  }
  // large systems are staged in a pinned buffer from the pool (the upload then runs at the
  // link's rate); small ones in ordinary memory, which many systems packed at once (batches)
  // would otherwise turn into pinned allocations
  void *hstage = nullptr;
  size_t hcap = 0;
  std::unique_ptr<char[]> small;
  char *host = nullptr;
  if (bytes >= ((size_t)4 << 20)) {
    VX_CHECK(pinned_get(bytes, &hstage, &hcap));
    host = (char *)hstage;
  } else {
    small.reset(new (std::nothrow) char[std::max<size_t>(bytes, 1)]);
    host = small.get();
    if (!host) {
      set_error("out of host memory");
      return VX_ENOMEM;
    }
  }
  // the coefficient blocks first in the staging buffer, packed in place (the way the layouts
  // were: on the host pool for large polynomials, a thread each for mid-sized ones)
  std::vector<size_t> coff(npoly);
  size_t off = 0;
  for (int f = 0; f < npoly; ++f) {
    coff[f] = off;
    off += al((size_t)hp[f].st[0].blk_in * sizeof(double2));
  }
  {
    std::vector<int> rcs(npoly, VX_OK);
    std::vector<std::string> msgs(npoly);
    auto one = [&](int f, int chunks) {
      rcs[f] = pack_coefs(k, F[f], hp[f], chi ? chi[f] : nullptr, (double2 *)(host + coff[f]), chunks);
      if (rcs[f] != VX_OK) msgs[f] = vx_last_error();
    };
    if (large) {
      for (int f = 0; f < npoly; ++f) one(f, F[f].nterms >= kPackSplitTerms ? pool_chunks : 1);
    } else if (npoly > 1 && terms >= 20000) {
      std::vector<std::thread> th;
      for (int f = 0; f < npoly; ++f) th.emplace_back([&, f] { one(f, 1); });
      for (auto &t : th) t.join();
    } else {
      for (int f = 0; f < npoly; ++f) one(f, 1);
    }
    for (int f = 0; f < npoly; ++f)
      if (rcs[f] != VX_OK) {
        pinned_put(hstage, hcap);
        set_error("%s", msgs[f].c_str());
        return rcs[f];
      }
  }
  vx_system *sys = new (std::nothrow) vx_system();
  if (!sys) {
    pinned_put(hstage, hcap);
    set_error("out of host memory");
    return VX_ENOMEM;
  }
  cudaStream_t s = as_stream(stream);
  int rc = dmalloc(&sys->mem, bytes, s);
  if (rc != VX_OK) {
    pinned_put(hstage, hcap);
    delete sys;
    return rc;
  }
  sys->stream = s;
  sys->bytes = bytes;
  sys->dev.k = k;
  sys->dev.npoly = npoly;
  for (int f = 0; f < npoly; ++f) sys->dev.rel[f] = (int8_t)(rel ? rel[f] : VX_EQ);
  sys->M.assign((size_t)npoly * (k + 1), 1);
  sys->exps.resize(npoly);
  sys->coefs.resize(npoly);
  sys->coefs_hi.resize(npoly);
  for (int f = 0; f < npoly && keep_host; ++f) {
    sys->exps[f].assign(F[f].exps, F[f].exps + (size_t)F[f].nterms * k);
    sys->coefs[f].assign(F[f].coefs, F[f].coefs + F[f].nterms);
    if (chi && chi[f]) sys->coefs_hi[f].assign(chi[f], chi[f] + F[f].nterms);
  }
  char *dbase = (char *)sys->mem;
  auto put = [&](const void *src, size_t n) -> void * {
    std::memcpy(host + off, src, n);
    void *d = dbase + off;
    off += al(n);
    return d;
  };
  auto reserve = [&](size_t n) -> void * {  // device space only, filled on the device
    void *d = dbase + off;
    off += al(n);
    return d;
  };
  for (int f = 0; f < npoly; ++f) {
    PolyDev &P = sys->dev.p[f];
    P.c64 = (const double2 *)(dbase + coff[f]);  // packed in place above
    for (int s2 = 0; s2 < k; ++s2) {
      const HostStage &S = hp[f].st[s2];
      StageDev &D = P.st[s2];
      D.nfib = S.nfib;
      D.maxlen = S.maxlen;
      D.blk_in = S.blk_in;
      D.blk_out = S.blk_out;
      D.rowoff = (const int32_t *)put(S.rowoff.data(), (S.maxlen + 1) * 4);
      D.fiblen = (const int32_t *)put(S.fiblen.data(), (size_t)S.nfib * 4);
      D.outpos = (const int32_t *)put(S.outpos.data(), (size_t)S.nfib * 4);
      D.fiboff = (const int32_t *)put(S.fiboff.data(), ((size_t)S.nfib + 1) * 4);
      D.outpos_fm = (const int32_t *)put(S.outpos_fm.data(), (size_t)S.nfib * 4);
      sys->M[(size_t)f * (k + 1) + s2] = S.blk_in;
    }
  }
  // the binary32 blocks are made on the device from the binary64 one (k_encode_coefs), after
  // everything that is uploaded: one copy of the prefix
  sys->upload_bytes = off;
  for (int f = 0; f < npoly; ++f) {
    PolyDev &P = sys->dev.p[f];
    const size_t nc = (size_t)hp[f].st[0].blk_in;
    P.c32 = (const float2 *)reserve(nc * sizeof(float2));
    P.c32c = (const float4 *)reserve(nc * sizeof(float4));
    P.c32c_fm = (const float4 *)reserve(nc * sizeof(float4));
    P.cp = (const float4 *)reserve(nc * sizeof(float4));
    P.ep = (const float *)reserve(nc * sizeof(float));
    P.cp_fm = (const float4 *)reserve(nc * sizeof(float4));
    P.ep_fm = (const float *)reserve(nc * sizeof(float));
    P.c64_fm = (const double2 *)reserve(nc * sizeof(double2));
    P.c32_fm = (const float2 *)reserve(nc * sizeof(float2));
  }
  cudaError_t e = cudaMemcpyAsync(sys->mem, host, sys->upload_bytes, cudaMemcpyHostToDevice, s);
  for (int f = 0; f < npoly && e == cudaSuccess; ++f) {
    const int64_t n = hp[f].st[0].blk_in;
    if (n == 0) continue;
    const int64_t nb = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    k_encode_coefs<<<(unsigned)nb, 256, 0, s>>>(sys->dev.p[f].c64,
                                                 n, const_cast<float2 *>(sys->dev.p[f].c32),
                                                 const_cast<float4 *>(sys->dev.p[f].c32c),
                                                 const_cast<float4 *>(sys->dev.p[f].cp),
                                                 const_cast<float *>(sys->dev.p[f].ep));
    note_launch();
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      const StageDev &S0 = sys->dev.p[f].st[0];
      const PolyDev &P = sys->dev.p[f];
      const Stage0Blocks r{P.c64, P.c32, P.c32c, P.cp, P.ep};
      const Stage0BlocksFm w{const_cast<double2 *>(P.c64_fm), const_cast<float2 *>(P.c32_fm),
                             const_cast<float4 *>(P.c32c_fm), const_cast<float4 *>(P.cp_fm),
                             const_cast<float *>(P.ep_fm)};
      k_fibre_major<<<(unsigned)std::min<int64_t>((S0.nfib + 3) / 4, (int64_t)sm_count() * 16),
                      128, 0, s>>>(r, S0.rowoff, S0.fiblen, S0.fiboff, S0.nfib, w);
      note_launch();
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  pinned_put(hstage, hcap);  // the copy has completed (or failed): the buffer is free again
  if (e != cudaSuccess) {
    set_error("uploading the system failed: %s", cudaGetErrorString(e));
    dfree(sys->mem, s);
    delete sys;
    return VX_ECUDA;
  }
  *out = sys;
  return VX_OK;
}

void vx_system_free(vx_system *sys) {
  if (!sys) return;
  for (auto &kv : sys->taylor)
    for (auto &ts : kv.second) vx_system_free(ts.sys);
  dfree(sys->mem, sys->stream);
  delete sys;
}

int vx_system_measure(const vx_poly *F, int32_t npoly, int64_t *h_M) {
  clear_error();
  if (!F || !h_M || npoly < 1 || npoly > VX_MAXPOLY) {
    set_error("vx_system_measure: need 1..%d polynomials and an output array", VX_MAXPOLY);
    return VX_EINVAL;
  }
  const int k = F[0].nvars;
  if (k < 1 || k > VX_KMAX) {
    set_error("vx_system_measure: %d variables (1..%d supported)", k, VX_KMAX);
    return VX_EINVAL;
  }
  const int pool_chunks = 2 * HostPool::get().size();
  for (int f = 0; f < npoly; ++f) {
    HostPoly hp;
    const int chunks = F[f].nterms >= kPackSplitTerms ? pool_chunks : 1;
    VX_CHECK(pack_poly(k, F[f], &hp, nullptr, chunks));
    // the coefficient block too, for its checks (a monomial given twice)
    std::vector<double2> blk((size_t)hp.st[0].blk_in);
    VX_CHECK(pack_coefs(k, F[f], hp, nullptr, blk.data(), chunks));
    for (int s2 = 0; s2 < k; ++s2) h_M[(size_t)f * (k + 1) + s2] = hp.st[s2].blk_in;
    h_M[(size_t)f * (k + 1) + k] = 1;
  }
  return VX_OK;
}

int vx_system_info(const vx_system *sys, int32_t *k, int32_t *npoly, int64_t *h_M) {
  clear_error();
  if (!sys) {
    set_error("vx_system_info: NULL system");
    return VX_EINVAL;
  }
  if (k) *k = sys->dev.k;
  if (npoly) *npoly = sys->dev.npoly;
  if (h_M) std::memcpy(h_M, sys->M.data(), sys->M.size() * sizeof(int64_t));
  return VX_OK;
}

int vx_system_device_bytes(const vx_system *sys, int64_t *bytes) {
  clear_error();
  if (!sys || !bytes) {
    set_error("vx_system_device_bytes: NULL argument");
    return VX_EINVAL;
  }
  *bytes = (int64_t)sys->bytes;
  return VX_OK;
}

int vx_system_upload_bytes(const vx_system *sys, int64_t *bytes) {
  clear_error();
  if (!sys || !bytes) {
    set_error("vx_system_upload_bytes: NULL argument");
    return VX_EINVAL;
  }
  *bytes = (int64_t)sys->upload_bytes;
  return VX_OK;
}

int64_t vx_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int vx_autotune(int32_t mode, const char *cache_path) {
  clear_error();
  if (mode < 0 || mode > 9) {
    set_error("vx_autotune: mode %d (0, 1, or 2 + a variant below 8)", mode);
    return VX_EINVAL;
  }
  return set_autotune(mode, cache_path);
}

int vx_autotune_entries(void) { return autotune_entries(); }

void vx_autotune_clear(void) { autotune_clear(); }

int vx_set_wait_limit(int64_t polls) {
  clear_error();
  VX_CHECK(set_dense_wait_polls(polls));
  return set_wait_polls(polls);
}

int vx_csf_build(int32_t k, int32_t level, const int32_t *d_tuples, int64_t n, void *stream,
                 vx_csf **out) {
  clear_error();
  if (!out || k < 1 || k > VX_KMAX || level < 0 || level > VX_MAXLEVEL || n < 0 ||
      (n > 0 && !d_tuples)) {
    set_error("vx_csf_build: bad arguments (k %d, level %d, n %lld)", k, level, (long long)n);
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_csf *c = new (std::nothrow) vx_csf();
  if (!c) return VX_ENOMEM;
  int rc = csf_build_dev(k, level, d_tuples, n, as_stream(stream), &c->o, nullptr);
  if (rc != VX_OK) {
    csf_release(&c->o);
    delete c;
    return rc;
  }
  *out = c;
  return VX_OK;
}

int vx_csf_full_grid(int32_t k, int32_t level, void *stream, vx_csf **out) {
  clear_error();
  if (!out || k < 1 || k > VX_KMAX || level < 0 || level > VX_MAXLEVEL) {
    set_error("vx_csf_full_grid: bad arguments (k %d, level %d)", k, level);
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_csf *c = new (std::nothrow) vx_csf();
  if (!c) return VX_ENOMEM;
  int rc = csf_full_grid_dev(k, level, as_stream(stream), &c->o);
  if (rc != VX_OK) {
    csf_release(&c->o);
    delete c;
    return rc;
  }
  *out = c;
  return VX_OK;
}

void vx_csf_free(vx_csf *c) {
  if (!c) return;
  csf_release(&c->o);
  delete c;
}

int vx_csf_nodes(const vx_csf *c, int32_t *k, int32_t *level, int64_t *h_N) {
  clear_error();
  if (!c) {
    set_error("vx_csf_nodes: NULL csf");
    return VX_EINVAL;
  }
  if (k) *k = c->o.v.k;
  if (level) *level = c->o.v.level;
  if (h_N)
    for (int d = 0; d < c->o.v.k; ++d) h_N[d] = c->o.v.N[d];
  return VX_OK;
}

int vx_csf_export(const vx_csf *c, int32_t depth, int32_t *d_labels, int32_t *d_ptr,
                  void *stream) {
  clear_error();
  if (!c || depth < 1 || depth > c->o.v.k || !d_labels) {
    set_error("vx_csf_export: bad arguments");
    return VX_EINVAL;
  }
  const int d = depth - 1;
  cudaStream_t s = as_stream(stream);
  const int64_t n = c->o.v.N[d];
  if (n > 0)
    VX_CUDA(cudaMemcpyAsync(d_labels, c->o.v.lab[d], n * 4, cudaMemcpyDeviceToDevice, s));
  if (d_ptr && d + 1 < c->o.v.k)
    VX_CUDA(cudaMemcpyAsync(d_ptr, c->o.v.ptr[d], (n + 1) * 4, cudaMemcpyDeviceToDevice, s));
  return VX_OK;
}

int vx_csf_tuples(const vx_csf *c, int32_t *d_tuples, void *stream) {
  clear_error();
  if (!c || (!d_tuples && c->o.v.N[c->o.v.k - 1] > 0)) {
    set_error("vx_csf_tuples: bad arguments");
    return VX_EINVAL;
  }
  return csf_tuples_dev(c->o.v, d_tuples, as_stream(stream));
}

int vx_csf_eval_level(const vx_system *sys, const vx_csf *c, const double *h_domain,
                      int32_t mode, double *d_lo, double *d_hi, uint8_t *d_keep, void *stream) {
  clear_error();
  if (!sys || !c || !d_keep || (mode != VX_FP64 && mode != VX_FP32_MIDRAD && mode != VX_FP32) ||
      (!d_lo) != (!d_hi) || c->o.v.k != sys->dev.k) {
    set_error("vx_csf_eval_level: bad arguments");
    return VX_EINVAL;
  }
  LevelGrid g;
  if (api_trace()) std::fprintf(stderr, "[vx] eval_level entry\n");
  VX_CHECK(make_grid(c->o.v.k, h_domain, c->o.v.level, &g));
  if (api_trace()) std::fprintf(stderr, "[vx] grid ok\n");
  int64_t w = 0, nr = 0;
  cudaStream_t s = as_stream(stream);
  VX_CHECK(eval_decide(sys->dev, c->o.v, g, mode, false, 0.5f, d_lo, d_hi, d_keep, s, nullptr, &w,
                       &nr));
  int st = 0;
  VX_CHECK(take_device_status(s, &st));
  if (st) {
    set_error("vx_csf_eval_level: a bounded device wait gave up; outputs are not valid");
    return VX_ETIMEOUT;
  }
  return VX_OK;
}

// ---------------------------------------------------------------------------------------
// Dense full-grid levels (tensor cores)
// ---------------------------------------------------------------------------------------
struct vx_dense_plan {
  DensePlan *p = nullptr;
  const vx_system *sys = nullptr;
  int level = 0;
  double domain[2 * VX_KMAX];
  uint32_t *mask = nullptr;  // vx_dense_level's mask (one address: the prefilter graph is reused)
  cudaStream_t stream = nullptr;
};

int vx_dense_plan_create(const vx_system *sys, int32_t level, const double *h_domain,
                         void *stream, vx_dense_plan **out) {
  clear_error();
  if (!sys || !h_domain || !out) {
    set_error("vx_dense_plan_create: bad arguments");
    return VX_EINVAL;
  }
  *out = nullptr;
  if (sys->dev.k != 3) {
    set_error("vx_dense_plan_create: the tensor-core level is for k = 3 (system has k = %d)",
              sys->dev.k);
    return VX_EINVAL;
  }
  for (int f = 0; f < sys->dev.npoly; ++f)
    if (sys->dev.rel[f] != VX_EQ || !sys->coefs_hi[f].empty()) {
      set_error("vx_dense_plan_create: equations with point coefficients only");
      return VX_EINVAL;
    }
  LevelGrid g;
  VX_CHECK(make_grid(3, h_domain, level, &g));  // the same domains as the interval path
  std::vector<DenseHostPoly> hp(sys->dev.npoly);
  for (int f = 0; f < sys->dev.npoly; ++f)
    hp[f] = DenseHostPoly{sys->exps[f].data(), sys->coefs[f].data(),
                          (int64_t)sys->coefs[f].size()};
  vx_dense_plan *d = new (std::nothrow) vx_dense_plan();
  if (!d) {
    set_error("out of host memory");
    return VX_ENOMEM;
  }
  d->sys = sys;
  d->level = level;
  d->stream = as_stream(stream);
  std::memcpy(d->domain, h_domain, 6 * sizeof(double));
  cudaStream_t s = as_stream(stream);
  int rc = dense_plan_create(sys->dev.npoly, hp.data(), level, h_domain, s, &d->p);
  if (rc == VX_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("vx_dense_plan_create: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  if (rc != VX_OK) {
    dense_plan_free(d->p);
    delete d;
    return rc;
  }
  *out = d;
  return VX_OK;
}

int vx_dense_plan_bytes(const vx_dense_plan *plan, int64_t *bytes) {
  clear_error();
  if (!plan || !bytes) {
    set_error("vx_dense_plan_bytes: bad arguments");
    return VX_EINVAL;
  }
  *bytes = dense_plan_bytes(plan->p);
  return VX_OK;
}

void vx_dense_plan_free(vx_dense_plan *plan) {
  if (!plan) return;
  dfree(plan->mask, plan->stream);
  dense_plan_free(plan->p);
  delete plan;
}

int vx_dense_prefilter(const vx_dense_plan *plan, uint32_t *d_mask, void *stream) {
  clear_error();
  if (!plan || !d_mask) {
    set_error("vx_dense_prefilter: bad arguments");
    return VX_EINVAL;
  }
  return dense_prefilter(plan->p, d_mask, as_stream(stream));
}

int vx_dense_check_status(void *stream) {
  clear_error();
  int st = 0;
  VX_CHECK(take_dense_status(as_stream(stream), &st));
  if (st) {
    set_error("a bounded wait in a tensor-core kernel gave up; its outputs are not valid");
    return VX_ETIMEOUT;
  }
  return VX_OK;
}

int vx_dense_values(const vx_dense_plan *plan, int32_t poly, float *d_mid, float *d_rad,
                    void *stream) {
  clear_error();
  if (!plan || !d_mid || !d_rad) {
    set_error("vx_dense_values: bad arguments");
    return VX_EINVAL;
  }
  VX_CHECK(dense_values(plan->p, poly, d_mid, d_rad, as_stream(stream)));
  return vx_dense_check_status(stream);
}

int vx_dense_level(const vx_dense_plan *plan, const vx_opts *opts, uint8_t *d_keep,
                   int64_t *n_survivors, void *stream) {
  clear_error();
  if (!plan || !d_keep) {
    set_error("vx_dense_level: bad arguments");
    return VX_EINVAL;
  }
  const int mode = opts ? opts->mode : VX_FP32;
  if (mode != VX_FP64 && mode != VX_FP32 && mode != VX_FP32_MIDRAD) {
    set_error("vx_dense_level: unknown mode %d", mode);
    return VX_EINVAL;
  }
  cudaStream_t s = as_stream(stream);
  const int level = plan->level;
  const int64_t nbox = (int64_t)1 << (3 * level);
  if (nbox > INT32_MAX) {
    set_error("vx_dense_level: %lld boxes exceed the 32-bit tree indices", (long long)nbox);
    return VX_EOVERFLOW;
  }
  LevelGrid g;
  VX_CHECK(make_grid(3, plan->domain, level, &g));
  int32_t *tup = nullptr;
  uint8_t *sub = nullptr;
  int64_t n = 0;
  int rc = VX_OK;
  vx_dense_plan *mp = const_cast<vx_dense_plan *>(plan);  // the plan's own mask, made once
  if (!mp->mask) rc = dmalloc((void **)&mp->mask, (size_t)(nbox / 8), s);
  uint32_t *mask = mp->mask;
  if (rc == VX_OK) rc = dense_prefilter(plan->p, mask, s);
  if (rc == VX_OK) rc = vx_dense_check_status(stream);
  if (rc == VX_OK) rc = mask_tuples(mask, level, s, &tup, &n);
  if (rc == VX_OK) {
    cudaError_t e = cudaMemsetAsync(d_keep, 0, (size_t)nbox, s);
    if (e != cudaSuccess) {
      set_error("vx_dense_level: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  if (rc == VX_OK && n > 0) {
    CsfObj c;
    rc = csf_build_dev(3, level, tup, n, s, &c, nullptr);
    if (rc == VX_OK) rc = dmalloc((void **)&sub, (size_t)n, s);
    int64_t w = 0, nr = 0;
    if (rc == VX_OK)
      rc = eval_decide(plan->sys->dev, c.v, g, mode, false, 0.5f, nullptr, nullptr, sub, s,
                       nullptr, &w, &nr);
    if (rc == VX_OK) rc = scatter_keep_grid(tup, n, level, sub, d_keep, s);
    csf_release(&c);
  }
  if (rc == VX_OK) {
    int st = 0;
    rc = take_device_status(s, &st);
    if (rc == VX_OK && st) {
      set_error("vx_dense_level: a bounded device wait gave up; outputs are not valid");
      rc = VX_ETIMEOUT;
    }
  }
  dfree(sub, s);
  dfree(tup, s);
  if (rc == VX_OK && n_survivors) *n_survivors = n;
  return rc;
}

// ---------------------------------------------------------------------------------------
// Taylor form (Def. 3): G_a = d^a F / a! = sum_e f_e prod_i binom(e_i, a_i) x^(e - a) for the
// multi-indices |a| <= m in lexicographic order; the coefficients become intervals
// [RD(f_e C), RU(f_e C)] (C an integer below 2^53, the product rounded both ways exactly).
// ---------------------------------------------------------------------------------------
static int taylor_sets(const vx_system *csys, int m, cudaStream_t s,
                       std::vector<vx_system::TaylorSet> **out) {
  vx_system *sys = const_cast<vx_system *>(csys);  // the cache is the system's own
  std::lock_guard<std::mutex> g(sys->tmu);
  auto it = sys->taylor.find(m);
  if (it != sys->taylor.end()) {
    *out = &it->second;
    return VX_OK;
  }
  const int k = sys->dev.k;
  std::vector<std::array<int8_t, VX_KMAX>> alpha;
  {
    int a[VX_KMAX] = {0};
    for (;;) {
      int tot = 0;
      for (int i = 0; i < k; ++i) tot += a[i];
      if (tot <= m) {
        std::array<int8_t, VX_KMAX> al{};
        for (int i = 0; i < k; ++i) al[i] = (int8_t)a[i];
        alpha.push_back(al);
      }
      int i = k - 1;
      while (i >= 0 && a[i] == m) a[i--] = 0;
      if (i < 0) break;
      ++a[i];
    }
  }
  if ((int)alpha.size() > VX_MAXPOLY) {
    set_error("Taylor form of order %d in %d variables has %zu terms (at most %d)", m, k,
              alpha.size(), VX_MAXPOLY);
    return VX_EINVAL;
  }
  std::vector<vx_system::TaylorSet> sets(sys->dev.npoly);
  int rc = VX_OK;
  for (int f = 0; f < sys->dev.npoly && rc == VX_OK; ++f) {
    const std::vector<int32_t> &E = sys->exps[f];
    const std::vector<double> &Cf = sys->coefs[f];
    const std::vector<double> &Ch = sys->coefs_hi[f].empty() ? Cf : sys->coefs_hi[f];
    const int64_t nt = (int64_t)Cf.size();
    const int na = (int)alpha.size();
    std::vector<std::vector<int32_t>> de(na);
    std::vector<std::vector<double>> lo(na), hi(na);
    for (int a = 0; a < na && rc == VX_OK; ++a)
      for (int64_t t = 0; t < nt; ++t) {
        bool ok = true;
        for (int i = 0; i < k; ++i) ok = ok && E[t * k + i] >= alpha[a][i];
        if (!ok) continue;
        double C = 1.0;
        for (int i = 0; i < k; ++i) {
          const int n = E[t * k + i], r = alpha[a][i];
          double b = 1.0;
          for (int j = 1; j <= r; ++j) b = b * (double)(n - r + j) / (double)j;  // exact integers
          C *= b;
        }
        if (C >= 9007199254740992.0) {
          set_error("Taylor form: a binomial product reaches 2^53");
          rc = VX_EINVAL;
          break;
        }
        const double c = Cf[t], p = c * C, err = std::fma(c, C, -p);
        const double ch = Ch[t], ph = ch * C, errh = std::fma(ch, C, -ph);
        lo[a].push_back(err < 0 ? std::nextafter(p, -INFINITY) : p);
        hi[a].push_back(errh > 0 ? std::nextafter(ph, INFINITY) : ph);
        for (int i = 0; i < k; ++i) de[a].push_back(E[t * k + i] - alpha[a][i]);
      }
    if (rc != VX_OK) break;
    std::vector<vx_poly> P(na);
    std::vector<const double *> chi(na);
    for (int a = 0; a < na; ++a) {
      P[a].nvars = k;
      P[a].nterms = (int32_t)lo[a].size();
      P[a].exps = de[a].empty() ? nullptr : de[a].data();
      P[a].coefs = lo[a].empty() ? nullptr : lo[a].data();
      chi[a] = hi[a].empty() ? nullptr : hi[a].data();
    }
    rc = system_create_impl(P.data(), na, chi.data(), (void *)s, &sets[f].sys);
    sets[f].alpha = alpha;
  }
  if (rc != VX_OK) {
    for (auto &ts : sets) vx_system_free(ts.sys);
    return rc;
  }
  auto ins = sys->taylor.emplace(m, std::move(sets));
  *out = &ins.first->second;
  return VX_OK;
}

static __global__ void k_and_flag(uint8_t *__restrict__ flag, const uint8_t *__restrict__ keep,
                                  int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    flag[i] = flag[i] & keep[i];
}

// One level with C0 on the Taylor form of order m (and C1 on it when inc is non-null), in
// VX_FP64 or in certified binary32 (VX_FP32): there the boxes whose decision binary32 cannot
// certify (and that no polynomial surely excludes) are gathered into a tree of their own,
// decided by the binary64 form, and their decisions scattered back, so every decision is the
// binary64 one.  d_lo/d_hi (binary64 only, nullable) receive the forms.
static int eval_taylor_level(const vx_system *sys, const CsfView &c, const LevelGrid &g, int m,
                             int mode, double *d_lo, double *d_hi, uint8_t *keep, uint8_t *inc,
                             cudaStream_t s, Timer *tm, int64_t *madds, int64_t *nrecheck) {
  for (int d = 0; d < c.k; ++d)  // the centres are points of the next level's grid
    if (!grid_exact(g.ax[d].lo, 0.5 * g.ax[d].w, (int64_t)2 << c.level, 53, -1074)) {
      set_error("axis %d: the box centres of level %d are not binary64 numbers", d, c.level);
      return VX_EINVAL;
    }
  if (inc && (sys->dev.npoly != 1 || sys->dev.rel[0] != VX_EQ)) {
    set_error("C1 is a test for one equation");
    return VX_EINVAL;
  }
  const bool cert = mode == VX_FP32;
  if ((mode != VX_FP64 && !cert) || (cert && d_lo)) {
    set_error("the Taylor form is evaluated in VX_FP64 or VX_FP32 (values in VX_FP64 only)");
    return VX_EINVAL;
  }
  std::vector<vx_system::TaylorSet> *sets = nullptr;
  VX_CHECK(taylor_sets(sys, m, s, &sets));
  const int64_t n = c.N[c.k - 1];
  *madds = 0;
  if (nrecheck) *nrecheck = 0;
  uint8_t *flag = nullptr;
  if (cert) VX_CHECK(dmalloc((void **)&flag, (size_t)std::max<int64_t>(n, 1), s));
  int rc = VX_OK;
  for (int f = 0; f < sys->dev.npoly && rc == VX_OK; ++f) {
    const vx_system::TaylorSet &ts = (*sets)[f];
    std::vector<int8_t> al((size_t)ts.alpha.size() * VX_KMAX);
    for (size_t a = 0; a < ts.alpha.size(); ++a)
      for (int d = 0; d < VX_KMAX; ++d) al[a * VX_KMAX + d] = ts.alpha[a][d];
    int64_t w = 0;
    rc = eval_level_taylor(ts.sys->dev, (const int8_t(*)[VX_KMAX])al.data(), m, c, g, keep, f == 0,
                           sys->dev.rel[f], d_lo ? d_lo + (int64_t)f * n : nullptr,
                           d_hi ? d_hi + (int64_t)f * n : nullptr, inc, flag, s, tm, &w);
    *madds += w;
  }
  if (rc == VX_OK && cert && n > 0) {
    // unsure and not surely excluded: the binary64 form decides
    k_and_flag<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(flag, keep, n);
    note_launch();
    int32_t *idx = nullptr, *tup = nullptr;
    uint8_t *subkeep = nullptr, *subinc = nullptr;
    int64_t ns = 0;
    rc = flag_indices(flag, n, s, &idx, &ns);
    if (nrecheck) *nrecheck = ns;
    if (rc == VX_OK && ns > 0) {
      CsfObj sub;
      const int k = c.k;
      rc = dmalloc((void **)&tup, (size_t)ns * k * 4, s);
      if (rc == VX_OK) rc = csf_tuples_of(c, idx, ns, tup, s);
      if (rc == VX_OK) rc = csf_build_dev(k, c.level, tup, ns, s, &sub, tm);
      if (rc == VX_OK) rc = dmalloc((void **)&subkeep, (size_t)ns, s);
      if (rc == VX_OK && inc) rc = dmalloc((void **)&subinc, (size_t)ns, s);
      int64_t w2 = 0;
      if (rc == VX_OK)
        rc = eval_taylor_level(sys, sub.v, g, m, VX_FP64, nullptr, nullptr, subkeep, subinc, s,
                               tm, &w2, nullptr);
      *madds += w2;
      if (rc == VX_OK) rc = scatter_keep(idx, subkeep, ns, keep, s);
      if (rc == VX_OK && inc) rc = scatter_keep(idx, subinc, ns, inc, s);
      csf_release(&sub);
    }
    dfree(subinc, s);
    dfree(subkeep, s);
    dfree(tup, s);
    dfree(idx, s);
  }
  dfree(flag, s);
  return rc;
}

int vx_csf_eval_level_taylor(const vx_system *sys, const vx_csf *c, const double *h_domain,
                             int32_t order, double *d_lo, double *d_hi, uint8_t *d_keep,
                             void *stream) {
  clear_error();
  if (!sys || !c || !d_keep || (!d_lo) != (!d_hi) || c->o.v.k != sys->dev.k || order < 1) {
    set_error("vx_csf_eval_level_taylor: bad arguments");
    return VX_EINVAL;
  }
  LevelGrid g;
  VX_CHECK(make_grid(c->o.v.k, h_domain, c->o.v.level, &g));
  cudaStream_t s = as_stream(stream);
  if (c->o.v.N[c->o.v.k - 1] == 0) return VX_OK;
  int64_t w = 0;
  VX_CHECK(eval_taylor_level(sys, c->o.v, g, order, VX_FP64, d_lo, d_hi, d_keep, nullptr, s,
                             nullptr, &w, nullptr));
  int st = 0;
  VX_CHECK(take_device_status(s, &st));
  if (st) {
    set_error("vx_csf_eval_level_taylor: a bounded device wait gave up");
    return VX_ETIMEOUT;
  }
  return VX_OK;
}

int vx_csf_taylor_level(const vx_system *sys, const vx_csf *c, const double *h_domain,
                        int32_t order, int32_t mode, uint8_t *d_keep, uint8_t *d_inc,
                        int64_t *n_recheck, void *stream) {
  clear_error();
  if (!sys || !c || !d_keep || c->o.v.k != sys->dev.k || order < 1 || (d_inc && order < 2)) {
    set_error("vx_csf_taylor_level: bad arguments");
    return VX_EINVAL;
  }
  LevelGrid g;
  VX_CHECK(make_grid(c->o.v.k, h_domain, c->o.v.level, &g));
  cudaStream_t s = as_stream(stream);
  if (n_recheck) *n_recheck = 0;
  if (c->o.v.N[c->o.v.k - 1] == 0) return VX_OK;
  int64_t w = 0;
  VX_CHECK(eval_taylor_level(sys, c->o.v, g, order, mode, nullptr, nullptr, d_keep, d_inc, s,
                             nullptr, &w, n_recheck));
  int st = 0;
  VX_CHECK(take_device_status(s, &st));
  if (st) {
    set_error("vx_csf_taylor_level: a bounded device wait gave up");
    return VX_ETIMEOUT;
  }
  VX_CUDA(cudaStreamSynchronize(s));
  return VX_OK;
}

int vx_csf_c1(const vx_system *sys, const vx_csf *c, const double *h_domain, int32_t kind,
              int32_t order, uint8_t *d_inc, void *stream) {
  clear_error();
  if (!sys || !c || !d_inc || c->o.v.k != sys->dev.k ||
      (kind != VX_C1_TAYLOR && kind != VX_C1_VERTEX) || (kind == VX_C1_TAYLOR && order < 2)) {
    set_error("vx_csf_c1: bad arguments");
    return VX_EINVAL;
  }
  if (sys->dev.npoly != 1 || sys->dev.rel[0] != VX_EQ) {
    set_error("vx_csf_c1: C1 is a test for one equation");
    return VX_EINVAL;
  }
  LevelGrid g;
  VX_CHECK(make_grid(c->o.v.k, h_domain, c->o.v.level, &g));
  cudaStream_t s = as_stream(stream);
  const int64_t n = c->o.v.N[c->o.v.k - 1];
  if (n == 0) return VX_OK;
  int64_t w = 0;
  int rc = VX_OK;
  if (kind == VX_C1_VERTEX) {
    rc = eval_c1_vertex(sys->dev, c->o.v, g, d_inc, s, nullptr, &w);
  } else {
    uint8_t *keep = nullptr;
    rc = dmalloc((void **)&keep, (size_t)n, s);
    if (rc == VX_OK) rc = eval_taylor_level(sys, c->o.v, g, order, VX_FP64, nullptr, nullptr, keep,
                                            d_inc, s, nullptr, &w, nullptr);
    dfree(keep, s);
  }
  int st = 0;
  if (rc == VX_OK) rc = take_device_status(s, &st);
  if (rc == VX_OK && st) {
    set_error("vx_csf_c1: a bounded device wait gave up");
    rc = VX_ETIMEOUT;
  }
  return rc;
}

int vx_csf_eval_grid(const vx_system *sys, const vx_csf *c, const double *const *d_xlo,
                     const double *const *d_xhi, const int64_t *nx, int32_t mode, double *d_lo,
                     double *d_hi, uint8_t *d_keep, void *stream) {
  clear_error();
  if (!sys || !c || !d_xlo || !d_xhi || !nx || !d_keep || (!d_lo) != (!d_hi) ||
      c->o.v.k != sys->dev.k || (mode != VX_FP64 && mode != VX_FP32_MIDRAD && mode != VX_FP32)) {
    set_error("vx_csf_eval_grid: bad arguments");
    return VX_EINVAL;
  }
  const int k = c->o.v.k;
  const int64_t side = (int64_t)1 << c->o.v.level;
  LevelGrid g{};
  for (int i = 0; i < k; ++i) {
    if (!d_xlo[i] || !d_xhi[i] || nx[i] < side) {
      set_error("vx_csf_eval_grid: axis %d needs %lld intervals (labels < 2^level), got %lld", i,
                (long long)side, (long long)nx[i]);
      return VX_EINVAL;
    }
    g.ax[i].xlo = d_xlo[i];
    g.ax[i].xhi = d_xhi[i];
    g.ax[i].fexact = 0;
  }
  int64_t w = 0, nr = 0;
  cudaStream_t s = as_stream(stream);
  VX_CHECK(eval_decide(sys->dev, c->o.v, g, mode, false, 0.5f, d_lo, d_hi, d_keep, s, nullptr, &w,
                       &nr));
  int st = 0;
  VX_CHECK(take_device_status(s, &st));
  if (st) {
    set_error("vx_csf_eval_grid: a bounded device wait gave up; outputs are not valid");
    return VX_ETIMEOUT;
  }
  return VX_OK;
}

int vx_csf_eval_level_static(const vx_system *sys, const vx_csf *c, const double *h_domain,
                             int32_t mode, double *d_lo, double *d_hi, uint8_t *d_keep,
                             void *stream) {
  clear_error();
  if (!sys || !c || !d_keep || (!d_lo) != (!d_hi) || c->o.v.k != sys->dev.k) {
    set_error("vx_csf_eval_level_static: bad arguments");
    return VX_EINVAL;
  }
  if (mode != VX_FP64 && mode != VX_FP32_MIDRAD) {
    set_error("vx_csf_eval_level_static: mode %d is not available without allocation (VX_FP32 "
              "re-evaluates boxes in trees of their own); use VX_FP64 or VX_FP32_MIDRAD", mode);
    return VX_EINVAL;
  }
  LevelGrid g;
  VX_CHECK(make_grid(c->o.v.k, h_domain, c->o.v.level, &g));
  cudaStream_t s = as_stream(stream);
  VX_CHECK(eval_level_static(sys->dev, c->o.v, g, mode == VX_FP64 ? ARITH_F64 : ARITH_F32_MIDRAD,
                             d_lo, d_hi, d_keep, s));
  int st = 0;
  VX_CHECK(take_device_status(s, &st));
  if (st) {
    set_error("vx_csf_eval_level_static: a bounded device wait gave up; outputs are not valid");
    return VX_ETIMEOUT;
  }
  return VX_OK;
}

int vx_csf_subdivide(const vx_csf *in, const uint8_t *d_keep, void *stream, vx_csf **out) {
  clear_error();
  if (!in || !out || (!d_keep && in->o.v.N[in->o.v.k - 1] > 0)) {
    set_error("vx_csf_subdivide: bad arguments");
    return VX_EINVAL;
  }
  if (in->o.v.level + 1 > VX_MAXLEVEL) {
    set_error("vx_csf_subdivide: level %d is the finest supported", in->o.v.level);
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_csf *c = new (std::nothrow) vx_csf();
  if (!c) return VX_ENOMEM;
  int rc = csf_prune(in->o.v, d_keep, 1, nullptr, as_stream(stream), &c->o, nullptr);
  if (rc != VX_OK) {
    csf_release(&c->o);
    delete c;
    return rc;
  }
  *out = c;
  return VX_OK;
}

int vx_csf_compact(const vx_csf *in, const uint8_t *d_keep, int32_t *d_index, void *stream,
                   vx_csf **out) {
  clear_error();
  if (!in || !out || (!d_keep && in->o.v.N[in->o.v.k - 1] > 0)) {
    set_error("vx_csf_compact: bad arguments");
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_csf *c = new (std::nothrow) vx_csf();
  if (!c) return VX_ENOMEM;
  int rc = csf_prune(in->o.v, d_keep, 0, d_index, as_stream(stream), &c->o, nullptr);
  if (rc != VX_OK) {
    csf_release(&c->o);
    delete c;
    return rc;
  }
  *out = c;
  return VX_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Algorithm 3: the level loop
// ---------------------------------------------------------------------------------------
static int level0(int k, cudaStream_t s, CsfObj *o) {
  int64_t N[VX_KMAX];
  for (int d = 0; d < VX_KMAX; ++d) N[d] = 1;
  VX_CHECK(csf_alloc(o, k, 0, N, s));
  // one box (0, ..., 0): labels 0, parents 0, child ranges [0, 1)
  VX_CUDA(cudaMemsetAsync(o->mem, 0, o->bytes, s));
  return set_ptr_sentinels(o->v, s);
}

static int csf_copy(const CsfObj &src, cudaStream_t s, CsfObj *dst) {
  VX_CHECK(csf_alloc(dst, src.v.k, src.v.level, src.v.N, s));
  // the same counts give the same layout inside the allocation
  VX_CUDA(cudaMemcpyAsync(dst->mem, src.mem, src.bytes, cudaMemcpyDeviceToDevice, s));
  return VX_OK;
}

// With C1: inc &= keep (the certified boxes among the C0 survivors), keep &= !inc (the boxes
// that go on being bisected).
static __global__ void k_c1_split(uint8_t *__restrict__ keep, uint8_t *__restrict__ inc,
                                  int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint8_t kp = keep[i], c = inc[i] & kp;
    inc[i] = c;
    keep[i] = kp & (uint8_t)(c ^ 1);
  }
}

// The state of one enclosure while its levels run (Algorithm 3).
struct EncloseRun {
  const vx_system *sys;
  const double *dom;
  int depth, k;
  vx_opts opts;
  float theta;
  cudaStream_t s;
  vx_result *R;
  Timer *tm;
  int64_t cap;  // the most boxes one tree may hold at a level (the leaves' count)
  bool chunked = false;  // the levels run in x_1 ranges (several final trees)
};

// CodesSink of the last level's compaction (opts.host_codes): a pinned pool buffer for the
// result's codes, which the device writes through its mapped address.
static int host_codes_get(void *ctx, int64_t n, int cb, void **d_codes) {
  vx_result *R = static_cast<vx_result *>(ctx);
  *d_codes = nullptr;
  void *hb = nullptr;
  size_t cap = 0;
  VX_CHECK(pinned_get((size_t)n * cb, &hb, &cap));
  void *dh = nullptr;
  if (cudaHostGetDevicePointer(&dh, hb, 0) != cudaSuccess || !dh) {
    cudaGetLastError();  // not device-addressable: vx_result_box_codes makes them later
    pinned_put(hb, cap);
    return VX_OK;
  }
  R->hcodes = hb;
  R->hcodes_cap = cap;
  R->hcodes_count = n;
  *d_codes = dh;
  return VX_OK;
}

static void result_append(vx_result *R, CsfObj &fin) {
  if (!R->fin_set) {
    R->fin = fin;
    R->fin_set = true;
  } else {
    R->more.push_back(fin);
  }
}

// Level l of Algorithm 3 on cur: C0 (and C1 from its level on); keep flags of the leaves
// (caller frees), the boxes C1 certified moved to R->incl.  With the vertex test, cur is
// replaced by its C0 survivors.
// *status_deferred: the device status of the level's evaluation was queued into status_word()
// instead of read (the caller reads it after its next wait on the stream).
static int level_step(EncloseRun &E, CsfObj &cur, int l, uint8_t **keep_out,
                      int64_t *included_out, bool *status_deferred) {
  const int k = E.k;
  const vx_opts &opts = E.opts;
  const cudaStream_t s = E.s;
  vx_result *R = E.R;
  Timer *tm = E.tm;
  *keep_out = nullptr;
  *included_out = 0;
  *status_deferred = false;
  LevelGrid g;
  VX_CHECK(make_grid(k, E.dom, l, &g));
  const int64_t n = cur.v.N[k - 1];
  R->tested[l] += n;
  for (int d = 0; d < k; ++d) R->nodes[(size_t)l * k + d] += cur.v.N[d];
  int mode = opts.mode;
  if (mode == VX_FP32_MIDRAD && opts.fp64_final && l == E.depth) mode = VX_FP64;
  if (mode == VX_FP32 && opts.small_level_madds > 0) {
    // Theorem 1's count for this level (every polynomial and depth), times the Taylor
    // form's derivatives: small levels run in binary64, which decides the same way
    int64_t w = 0;
    for (int f = 0; f < E.sys->dev.npoly; ++f)
      for (int d = 0; d < k; ++d)
        w += cur.v.N[d] * (E.sys->dev.p[f].st[d].blk_in - E.sys->dev.p[f].st[d].nfib);
    if (opts.taylor_order > 0) {
      int64_t na = 1;  // C(m + k, k)
      for (int i = 1; i <= k; ++i) na = na * (opts.taylor_order + i) / i;
      w *= na;
    }
    if (w < opts.small_level_madds) mode = VX_FP64;
  }
  const bool c1_here = opts.c1 != 0 && l >= opts.c1_level && n > 0;
  uint8_t *keep = nullptr, *inc = nullptr;
  int rc = dmalloc((void **)&keep, (size_t)std::max<int64_t>(n, 1), s);
  if (rc == VX_OK && c1_here) rc = dmalloc((void **)&inc, (size_t)n, s);
  if (rc == VX_OK) {
    int64_t w = 0, nr = 0, nr64 = 0;
    if (opts.taylor_order > 0)
      rc = n > 0 ? eval_taylor_level(E.sys, cur.v, g, opts.taylor_order, mode, nullptr, nullptr,
                                     keep, opts.c1 == VX_C1_TAYLOR ? inc : nullptr, s, tm, &w,
                                     &nr)
                 : VX_OK;
    else
      rc = eval_decide(E.sys->dev, cur.v, g, mode, opts.fp64_recheck != 0, E.theta, nullptr,
                       nullptr, keep, s, tm, &w, &nr, opts.recheck_last != 0 && l < E.depth,
                       &nr64);
    R->madds[l] += w;
    R->recheck[l] += nr;
    R->recheck64[l] += mode == VX_FP32 ? nr64 : nr;
    int st = 0;
    int *hw = (!c1_here && n > 0) ? status_word() : nullptr;
    if (rc == VX_OK && hw) {  // read with the prune's wait that follows
      *hw = 0;
      rc = queue_device_status(s, hw);
      *status_deferred = rc == VX_OK;
    } else if (rc == VX_OK) {
      rc = take_device_status(s, &st);
    }
    if (rc == VX_OK && st) {
      set_error("enclose: a bounded device wait gave up at level %d", l);
      rc = VX_ETIMEOUT;
    }
  }
  int64_t included = 0;
  if (rc == VX_OK && c1_here) {
    // Algorithm 3's inclusion step: the C0 survivors that C1 certifies leave S
    int64_t nc = n;
    if (opts.c1 == VX_C1_VERTEX) {  // the corners are evaluated on the survivors only
      CsfObj surv;
      rc = csf_prune(cur.v, keep, 0, nullptr, s, &surv, tm);
      if (rc == VX_OK) {
        csf_release(&cur);
        cur = surv;
        nc = cur.v.N[k - 1];
        if (nc > 0) {
          const cudaError_t e = cudaMemsetAsync(keep, 1, (size_t)nc, s);
          if (e != cudaSuccess) {
            set_error("enclose: %s", cudaGetErrorString(e));
            rc = VX_ECUDA;
          }
        }
        if (rc == VX_OK && nc > 0) {
          int64_t w = 0;
          rc = eval_c1_vertex(E.sys->dev, cur.v, g, inc, s, tm, &w);
          R->madds[l] += w;
        }
      }
    }
    if (rc == VX_OK && nc > 0) {
      k_c1_split<<<(int)std::min<int64_t>((nc + 255) / 256, 4096), 256, 0, s>>>(keep, inc, nc);
      note_launch();
      CsfObj ic;
      rc = csf_prune(cur.v, inc, 0, nullptr, s, &ic, tm);
      if (rc == VX_OK) {
        included = ic.v.N[k - 1];
        if (included > 0) {
          try {
            R->incl.emplace_back(l, ic);
          } catch (...) {
            csf_release(&ic);
            set_error("enclose: out of host memory");
            rc = VX_ENOMEM;
          }
        } else {
          csf_release(&ic);
        }
      }
    }
  }
  dfree(inc, s);
  if (rc != VX_OK) {
    dfree(keep, s);
    return rc;
  }
  *keep_out = keep;
  *included_out = included;
  return VX_OK;
}

static int run_levels(EncloseRun &E, CsfObj &cur, int l);

// Level l's kept leaves would give the next level more than E.cap boxes in one tree: the kept
// boxes are split into runs of consecutive x_1 slabs (depth-0 nodes) whose children fit, and
// each run goes through the remaining levels on its own, in x_1 order.  A box's descendants
// stay in its slab and every box is decided on its own, so the runs' final boxes, one after
// another, are the enclosure's, in lexicographic order.
static int run_chunked(EncloseRun &E, CsfObj &cur, const uint8_t *keep, int l) {
  E.chunked = true;
  const int k = E.k;
  const cudaStream_t s = E.s;
  const int64_t n0 = cur.v.N[0], n = cur.v.N[k - 1];
  int64_t *d_cnt = nullptr;
  uint8_t *part = nullptr;
  std::vector<int64_t> cnt((size_t)std::max<int64_t>(n0, 1), 0);
  int rc = dmalloc((void **)&d_cnt, sizeof(int64_t) * cnt.size(), s);
  if (rc == VX_OK) rc = csf_root_counts(cur.v, keep, d_cnt, s);
  if (rc == VX_OK) {
    cudaError_t e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int64_t) * (size_t)n0,
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("enclose: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
  }
  dfree(d_cnt, s);
  int64_t total = 0;
  for (int64_t r = 0; r < n0; ++r) total += cnt[r];
  E.R->kept[l] += total;
  if (rc == VX_OK) rc = dmalloc((void **)&part, (size_t)std::max<int64_t>(n, 1), s);
  int64_t a = 0;
  while (rc == VX_OK && a < n0) {
    if ((cnt[a] << k) > E.cap) {
      set_error("enclose: one x1 slab at level %d has %lld kept boxes, whose children exceed "
                "the %lld boxes a level may hold", l, (long long)cnt[a], (long long)E.cap);
      rc = VX_EOVERFLOW;
      break;
    }
    int64_t b = a, acc = 0;
    while (b < n0 && ((acc + cnt[b]) << k) <= E.cap) acc += cnt[b++];
    if (acc > 0) {
      rc = csf_keep_in_roots(cur.v, keep, a, b, part, s);
      CsfObj next;
      if (rc == VX_OK) rc = csf_prune(cur.v, part, 1, nullptr, s, &next, E.tm, E.cap);
      if (rc == VX_OK) rc = run_levels(E, next, l + 1);  // consumes next
    }
    a = b;
  }
  dfree(part, s);
  return rc;
}

// Levels l..depth of Algorithm 3 from the tree cur (consumed); the final boxes are appended to
// the result.
static int run_levels(EncloseRun &E, CsfObj &cur, int l) {
  const int k = E.k;
  int rc = VX_OK;
  for (; l <= E.depth && rc == VX_OK; ++l) {
    uint8_t *keep = nullptr;
    int64_t included = 0;
    bool deferred = false;
    rc = level_step(E, cur, l, &keep, &included, &deferred);
    if (rc != VX_OK) break;
    // the level's device status, queued by level_step: the prune (n > 0) waits on the stream
    // for its counts, after which the word is in place; otherwise wait for it here
    auto status_after_prune = [&](int rc0) -> int {
      if (!deferred || (rc0 == VX_OK && *status_word() == 0)) return rc0;
      int st = 0;
      const int r = take_device_status(E.s, &st);
      if (r != VX_OK) return r;
      if (st) {
        set_error("enclose: a bounded device wait gave up at level %d", l);
        return VX_ETIMEOUT;
      }
      return rc0;
    };
    if (l == E.depth) {
      CsfObj fin;
      // the final boxes' codes straight to the host, where they will be one tree
      const CodesSink sink{host_codes_get, E.R};
      const bool eager = E.opts.host_codes && !E.chunked && !E.R->fin_set && E.R->hcodes_count < 0;
      const int rp = csf_prune(cur.v, keep, 0, nullptr, E.s, &fin, E.tm, INT32_MAX,
                               eager ? &sink : nullptr);
      rc = status_after_prune(rp);
      if (rp == VX_OK && rc != VX_OK) csf_release(&fin);
      if (rc == VX_OK) {
        E.R->kept[l] += fin.v.N[k - 1] + included;
        result_append(E.R, fin);
      }
    } else {
      CsfObj next;
      const int rp = csf_prune(cur.v, keep, 1, nullptr, E.s, &next, E.tm, E.cap);
      rc = status_after_prune(rp);
      if (rp == VX_OK && rc != VX_OK) csf_release(&next);
      if (rc == VX_EOVERFLOW && E.opts.c1 == 0) {
        // the next level does not fit one tree: run it in x_1 ranges
        clear_error();
        rc = run_chunked(E, cur, keep, l);
        dfree(keep, E.s);
        csf_release(&cur);
        return rc;
      }
      if (rc == VX_OK) {
        E.R->kept[l] += (next.v.N[k - 1] >> k) + included;
        csf_release(&cur);
        cur = next;
      }
    }
    dfree(keep, E.s);
  }
  csf_release(&cur);
  return rc;
}

static int enclose_impl(const vx_system *sys, const double *dom, int depth, const vx_opts *o,
                        cudaStream_t s, vx_result *R, const CsfObj *start) {
  const int k = sys->dev.k;
  vx_opts opts{};
  if (o) opts = *o;
  if (opts.mode != VX_FP64 && opts.mode != VX_FP32_MIDRAD && opts.mode != VX_FP32) {
    set_error("vx_enclose: unknown mode %d", opts.mode);
    return VX_EINVAL;
  }
  float theta = opts.theta > 0.f ? opts.theta : 0.5f;
  if (theta > 1.f) {
    set_error("vx_enclose: theta %g outside (0, 1]", (double)theta);
    return VX_EINVAL;
  }
  if (opts.taylor_order < 0 ||
      (opts.taylor_order > 0 && opts.mode != VX_FP64 && opts.mode != VX_FP32)) {
    set_error("vx_enclose: the Taylor form (order %d) is evaluated in VX_FP64 or VX_FP32",
              opts.taylor_order);
    return VX_EINVAL;
  }
  if (depth < 0 || depth > VX_MAXLEVEL) {
    set_error("vx_enclose: depth %d outside [0, %d]", depth, VX_MAXLEVEL);
    return VX_EINVAL;
  }
  if (opts.c1 != 0) {
    if (opts.c1 != VX_C1_TAYLOR && opts.c1 != VX_C1_VERTEX) {
      set_error("vx_enclose: unknown inclusion criterion %d", opts.c1);
      return VX_EINVAL;
    }
    if ((opts.mode != VX_FP64 && opts.mode != VX_FP32) || sys->dev.npoly != 1 ||
        sys->dev.rel[0] != VX_EQ || opts.c1_level < 0 ||
        (opts.c1 == VX_C1_TAYLOR && opts.taylor_order < 2)) {
      set_error("vx_enclose: C1 needs one equation, VX_FP64 or VX_FP32, c1_level >= 0 and, "
                "for VX_C1_TAYLOR, taylor_order >= 2");
      return VX_EINVAL;
    }
  }
  if (opts.first_level < 0 || (opts.first_level > 0 && (opts.taylor_order != 0 || opts.c1 != 0))) {
    set_error("vx_enclose: first_level %d needs the interval form (no Taylor form, no C1)",
              opts.first_level);
    return VX_EINVAL;
  }
  if (opts.first_level > 0) {
    int64_t n = 1;
    for (int i = 0; i < k; ++i) n <<= std::min<int>(opts.first_level, depth);
    if (n > INT32_MAX) {
      set_error("vx_enclose: the full grid of level %d has more than 2^31 - 1 boxes",
                opts.first_level);
      return VX_EINVAL;
    }
  }
  if (opts.recheck_last != 0 &&
      (opts.mode != VX_FP32 || opts.taylor_order != 0 || opts.c1 != 0)) {
    // the Taylor form is centred on each box, hence not inclusion-isotone across levels
    set_error("vx_enclose: recheck_last needs VX_FP32 on the interval form (no Taylor form, "
              "no C1)");
    return VX_EINVAL;
  }
  LevelGrid g;
  VX_CHECK(make_grid(k, dom, depth, &g));  // the finest grid exact => every coarser one too
  R->k = k;
  R->depth = depth;
  R->tested.assign(depth + 1, 0);
  R->kept.assign(depth + 1, 0);
  R->nodes.assign((size_t)(depth + 1) * k, 0);
  R->recheck.assign(depth + 1, 0);
  R->recheck64.assign(depth + 1, 0);
  R->madds.assign(depth + 1, 0);
  R->tm.on = opts.timing != 0;
  R->tm.stream = s;
  Timer *tm = &R->tm;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  VX_CUDA(cudaEventCreate(&ev0));
  VX_CUDA(cudaEventCreate(&ev1));
  VX_CUDA(cudaEventRecord(ev0, s));
  CsfObj cur;
  int rc = VX_OK;
  int l0 = 0;
  if (start) {
    if (start->v.k != k || start->v.level > depth) {
      set_error("enclose: the start tree has k = %d, level %d (system k = %d, depth %d)",
                start->v.k, start->v.level, k, depth);
      rc = VX_EINVAL;
    } else {
      l0 = start->v.level;
      rc = csf_copy(*start, s, &cur);
    }
  } else if (opts.first_level > 0) {
    // Algorithm 3 from the full grid of level first_level: the coarser levels' pruning does
    // not change the final boxes (C0 on interval Horner is inclusion-isotone over exact grids)
    l0 = std::min<int>(opts.first_level, depth);
    rc = csf_full_grid_dev(k, l0, s, &cur);
  } else {
    rc = level0(k, s, &cur);
  }
  if (rc == VX_OK) {
    EncloseRun E{sys, dom, depth, k, opts, theta, s, R, tm,
                 opts.max_level_boxes > 0 ? (int64_t)opts.max_level_boxes : (int64_t)INT32_MAX};
    rc = run_levels(E, cur, l0);  // consumes cur
  } else {
    csf_release(&cur);
  }
  if (rc == VX_OK) {
    cudaError_t e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e != cudaSuccess) {
      set_error("enclose: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
    R->elapsed_ms = ms;
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (rc == VX_OK) rc = R->tm.collect();
  return rc;
}

static cudaStream_t library_stream() {
  static cudaStream_t s = nullptr;
  static bool made = false;
  if (!made) {
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) s = nullptr;
    made = true;
  }
  return s;
}

extern "C" {

int vx_enclose_system(const vx_system *sys, const double *h_domain, int32_t depth,
                      const vx_opts *opts, void *stream, vx_result **out) {
  clear_error();
  if (!sys || !out) {
    set_error("vx_enclose_system: NULL argument");
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_result *R = new (std::nothrow) vx_result();
  if (!R) return VX_ENOMEM;
  int rc = enclose_impl(sys, h_domain, depth, opts, as_stream(stream), R, nullptr);
  if (rc != VX_OK) {
    result_release_trees(R);
    R->tm.release();
    delete R;
    return rc;
  }
  *out = R;
  return VX_OK;
}

int vx_enclose_from(const vx_system *sys, const vx_csf *start, const double *h_domain,
                    int32_t depth, const vx_opts *opts, void *stream, vx_result **out) {
  clear_error();
  if (!sys || !start || !out) {
    set_error("vx_enclose_from: NULL argument");
    return VX_EINVAL;
  }
  *out = nullptr;
  vx_result *R = new (std::nothrow) vx_result();
  if (!R) return VX_ENOMEM;
  int rc = enclose_impl(sys, h_domain, depth, opts, as_stream(stream), R, &start->o);
  if (rc != VX_OK) {
    result_release_trees(R);
    R->tm.release();
    delete R;
    return rc;
  }
  *out = R;
  return VX_OK;
}

int vx_enclose(const vx_poly *F, int32_t npoly, const double *h_domain, int32_t depth,
               const vx_opts *opts, vx_result **out) {
  clear_error();
  if (!out) {
    set_error("vx_enclose: NULL out");
    return VX_EINVAL;
  }
  *out = nullptr;
  cudaStream_t s = library_stream();
  vx_system *sys = nullptr;
  // the system lives for this call only: the host copy of the polynomials serves only the
  // Taylor form's derived system
  VX_CHECK(system_create_impl(F, npoly, nullptr, (void *)s, &sys, nullptr,
                              opts && opts->taylor_order > 0));
  int rc = vx_enclose_system(sys, h_domain, depth, opts, (void *)s, out);
  vx_system_free(sys);
  return rc;
}

// ---------------------------------------------------------------------------------------
// Batches (config 4): the systems with the same k go through Algorithm 3 together, as one
// forest of CSF trees per level.  Every depth of a level is one launch over every tree's
// nodes (eval_forest), and the prune and bisection are one multi-channel scan over the whole
// forest (csf_prune_forest), whose per-tree counts place each tree's nodes in the next
// forest: one host synchronisation per level and prune for all the systems.
// ---------------------------------------------------------------------------------------
namespace vx {
namespace {

// mode 0: out = keep && depth(tree) == l; 1: out = keep && depth(tree) > l;
// 2: out = out || (keep && depth(tree) == l) (the binary64 final level of VX_FP32_MIDRAD: a
// box the midpoint-radius superset drops, binary64 drops too); 3: out = out && depth(tree) == l
// (recheck_last: only the finishing trees' band is re-decided)
__global__ void k_tree_mask(const uint8_t *__restrict__ keep, const int64_t *__restrict__ offl,
                            int S, const int32_t *__restrict__ tdepth, int l, int mode,
                            int64_t n, uint8_t *__restrict__ out) {
  // 16 consecutive leaves per thread: one search for the tree of the first, then a walk
  // forward over the trees' boundaries (offl ascending)
  const int64_t nchunk = (n + 15) >> 4;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nchunk;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = q << 4, i1 = i0 + 16 < n ? i0 + 16 : n;
    int t = 0, hi = S;
    while (hi - t > 1) {
      const int mid = (t + hi) >> 1;
      if (__ldg(offl + mid) <= i0) t = mid; else hi = mid;
    }
    int64_t tend = __ldg(offl + t + 1);
    // a full chunk of 16-byte aligned arrays moves as one 16-byte load / store
    const bool full =
        i1 - i0 == 16 && ((reinterpret_cast<uintptr_t>(keep) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    if (full && i1 <= tend) {  // the whole chunk in tree t: one test, bytewise 0/1 logic
      const int dep = __ldg(tdepth + t);
      const bool c = mode == 1 ? dep > l : dep == l;
      const uint4 kv4 = *reinterpret_cast<const uint4 *>(keep + i0);
      uint4 r = make_uint4(0u, 0u, 0u, 0u);
      if (mode == 0 || mode == 1) {
        if (c) r = kv4;
      } else {
        const uint4 ov4 = *reinterpret_cast<const uint4 *>(out + i0);
        if (mode == 2)
          r = c ? make_uint4(ov4.x | kv4.x, ov4.y | kv4.y, ov4.z | kv4.z, ov4.w | kv4.w) : ov4;
        else if (c)
          r = ov4;
      }
      *reinterpret_cast<uint4 *>(out + i0) = r;
      continue;
    }
    alignas(16) uint8_t kv[16], ov[16];
    if (full) {
      *reinterpret_cast<uint4 *>(kv) = *reinterpret_cast<const uint4 *>(keep + i0);
      if (mode >= 2) *reinterpret_cast<uint4 *>(ov) = *reinterpret_cast<const uint4 *>(out + i0);
    }
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int64_t i = i0 + j;
      if (i >= i1) break;
      while (i >= tend && t + 1 < S) tend = __ldg(offl + (++t) + 1);
      const int dep = __ldg(tdepth + t);
      const bool kp = (full ? kv[j] : keep[i]) != 0;
      const bool o = mode >= 2 && (full ? ov[j] : out[i]) != 0;
      uint8_t r;
      if (mode == 0) r = (kp && dep == l) ? 1 : 0;
      else if (mode == 1) r = (kp && dep > l) ? 1 : 0;
      else if (mode == 2) r = (o || (kp && dep == l)) ? 1 : 0;
      else r = (o && dep == l) ? 1 : 0;
      if (full) ov[j] = r; else out[i] = r;
    }
    if (full) *reinterpret_cast<uint4 *>(out + i0) = *reinterpret_cast<const uint4 *>(ov);
  }
}

// Tree t of a forest as a CSF of its own: depth d copies nodes o[d] .. o[d]+n[d]-1, with
// parent and child indices rebased to the tree's own arrays.
struct TreeSlice {
  int64_t o[VX_KMAX], n[VX_KMAX];
};
__global__ void k_tree_extract(CsfView f, TreeSlice ts, CsfView out) {
  const int k = f.k;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int d = 0; d < k; ++d)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= ts.n[d]; i += stride) {
      if (i < ts.n[d]) {
        out.lab[d][i] = f.lab[d][ts.o[d] + i];
        if (d > 0) out.par[d][i] = (int32_t)(f.par[d][ts.o[d] + i] - ts.o[d - 1]);
      }
      if (d + 1 < k) out.ptr[d][i] = (int32_t)(f.ptr[d][ts.o[d] + i] - ts.o[d + 1]);
    }
}

__global__ void k_forest_level0(CsfView c, int S) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j <= S;
       j += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d < c.k; ++d) {
      if (j < S) {
        c.lab[d][j] = 0;
        if (d > 0) c.par[d][j] = (int32_t)j;
      }
      if (d + 1 < c.k) c.ptr[d][j] = (int32_t)j;
    }
}

int dmalloc_copy_trees(ForestTree *d_trees, const std::vector<ForestTree> &ht, cudaStream_t s) {
  // from pageable memory: returns once staged
  VX_CUDA(cudaMemcpyAsync(d_trees, ht.data(), sizeof(ForestTree) * ht.size(),
                          cudaMemcpyHostToDevice, s));
  return VX_OK;
}

// The level's grids into the device trees (the systems' part of a tree does not change
// between levels): the grids travel as one small array, a kernel puts them in place.
__global__ void k_set_tree_grids(ForestTree *__restrict__ trees, const AxisGrid *__restrict__ ax,
                                 int S) {
  const int n = S * VX_KMAX;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    trees[i / VX_KMAX].ax[i % VX_KMAX] = ax[i];
}

int copy_tree_grids(ForestTree *d_trees, AxisGrid *d_ax, const std::vector<ForestTree> &ht,
                    cudaStream_t s) {
  std::vector<AxisGrid> ax(ht.size() * VX_KMAX);
  for (size_t t = 0; t < ht.size(); ++t)
    for (int d = 0; d < VX_KMAX; ++d) ax[t * VX_KMAX + d] = ht[t].ax[d];
  // from pageable memory: returns once staged
  VX_CUDA(cudaMemcpyAsync(d_ax, ax.data(), sizeof(AxisGrid) * ax.size(), cudaMemcpyHostToDevice,
                          s));
  const int S = (int)ht.size();
  k_set_tree_grids<<<(S * VX_KMAX + 255) / 256, 256, 0, s>>>(d_trees, d_ax, S);
  note_launch();
  VX_CUDA(cudaGetLastError());
  return VX_OK;
}

int grid1(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sm_count() * 16) b = (int64_t)sm_count() * 16;
  return (int)std::max<int64_t>(b, 1);
}

struct Forest {
  CsfObj c;
  std::vector<int64_t> off;  // [k][S+1] host
  int64_t *d_off = nullptr;  // device copy
};

int upload_off(Forest &F, int k, int S, cudaStream_t s) {
  if (!F.d_off) VX_CHECK(dmalloc((void **)&F.d_off, sizeof(int64_t) * (size_t)k * (S + 1), s));
  VX_CUDA(cudaMemcpyAsync(F.d_off, F.off.data(), sizeof(int64_t) * (size_t)k * (S + 1),
                          cudaMemcpyHostToDevice, s));
  return VX_OK;
}

void release(Forest &F, cudaStream_t s) {
  csf_release(&F.c);
  dfree(F.d_off, s);
  F.d_off = nullptr;
}

// Prunes forest `in` with mask `m` (split or compact) into `out`, with per-tree offsets.
int prune_forest(Forest &in, const uint8_t *m, int split, int32_t *d_index, int k, int S,
                 int64_t *d_seg, std::vector<int64_t> &h_seg, cudaStream_t s, Forest &out) {
  h_seg.assign((size_t)k * (S + 1), 0);
  VX_CHECK(csf_prune_forest(in.c.v, m, split, d_index, in.d_off, S, d_seg, s, &out.c, nullptr,
                            h_seg.data()));
  out.off.assign(h_seg.size(), 0);
  for (int d = 0; d < k; ++d)
    for (int t = 0; t <= S; ++t)
      out.off[(size_t)d * (S + 1) + t] = h_seg[(size_t)d * (S + 1) + t] << (split ? d + 1 : 0);
  return upload_off(out, k, S, s);
}

int batch_group(const std::vector<int32_t> &ids, const vx_poly *const *systems,
                const int32_t *npoly, const double *domains, const std::vector<int64_t> &doff,
                const int32_t *depths, const vx_opts &opts, cudaStream_t s, vx_result **out) {
  const int S = (int)ids.size();
  const int k = systems[ids[0]][0].nvars;
  const float theta = opts.theta > 0.f ? opts.theta : 0.5f;
  std::vector<vx_system *> sysv(S, nullptr);
  std::vector<ForestTree> ht(S);
  std::vector<int32_t> tdep(S);
  int maxdepth = 0, rc = VX_OK;
  for (int t = 0; t < S && rc == VX_OK; ++t) {
    const int i = ids[t];
    if (depths[i] < 0 || depths[i] > VX_MAXLEVEL) {
      set_error("system %d: depth %d outside [0, %d]", i, depths[i], VX_MAXLEVEL);
      rc = VX_EINVAL;
      break;
    }
    tdep[t] = depths[i];
    maxdepth = std::max(maxdepth, depths[i]);
    LevelGrid g;
    rc = make_grid(k, domains + doff[i], depths[i], &g);  // the finest grid exact => all coarser
  }
  // packing is host work: host threads pack and upload the systems, each on a stream of its
  // own; the forest then reads them on `s`
  if (rc == VX_OK) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) rc = VX_ECUDA;
    const int nthr = std::max(1, std::min<int>(16, S));
    std::atomic<int> next{0}, first{VX_OK};
    std::vector<std::string> errs(nthr);
    auto work = [&](int w) {
      cudaStream_t ws = nullptr;
      if (cudaSetDevice(dev) != cudaSuccess ||
          cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking) != cudaSuccess) {
        first = VX_ECUDA;
        return;
      }
      for (int t = next++; t < S && first.load() == VX_OK; t = next++) {
        // no host copy of the polynomials: a batch has no Taylor form or dense plan
        const int r = system_create_impl(systems[ids[t]], npoly[ids[t]], nullptr, (void *)ws,
                                         &sysv[t], nullptr, false);
        if (r != VX_OK) {
          errs[w] = std::string("system ") + std::to_string(ids[t]) + ": " + vx_last_error();
          int expected = VX_OK;
          first.compare_exchange_strong(expected, r);
        } else {
          sysv[t]->stream = s;  // synchronised already; freed in the order of `s`
        }
      }
      cudaStreamDestroy(ws);
    };
    if (rc == VX_OK) {
      std::vector<std::thread> pool;
      for (int w = 0; w < nthr; ++w) pool.emplace_back(work, w);
      for (auto &th : pool) th.join();
      rc = first.load();
      if (rc != VX_OK)
        for (auto &e : errs)
          if (!e.empty()) {
            set_error("%s", e.c_str());
            break;
          }
    }
    for (int t = 0; t < S && rc == VX_OK; ++t) ht[t].dev = sysv[t]->dev;
  }
  ForestTree *d_trees = nullptr;
  AxisGrid *d_ax = nullptr;
  int32_t *d_tdep = nullptr;
  int64_t *d_seg = nullptr;
  if (rc == VX_OK) rc = dmalloc((void **)&d_trees, sizeof(ForestTree) * S, s);
  if (rc == VX_OK) rc = dmalloc((void **)&d_ax, sizeof(AxisGrid) * S * VX_KMAX, s);
  if (rc == VX_OK) rc = dmalloc((void **)&d_tdep, sizeof(int32_t) * S, s);
  if (rc == VX_OK) rc = dmalloc((void **)&d_seg, sizeof(int64_t) * (size_t)k * (S + 1), s);
  if (rc == VX_OK) {
    cudaError_t e = cudaMemcpyAsync(d_tdep, tdep.data(), sizeof(int32_t) * S,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = VX_ECUDA;
  }
  std::vector<vx_result *> R(S, nullptr);
  for (int t = 0; t < S && rc == VX_OK; ++t) {
    R[t] = new (std::nothrow) vx_result();
    if (!R[t]) {
      set_error("out of host memory");
      rc = VX_ENOMEM;
      break;
    }
    const int D = tdep[t];
    R[t]->k = k;
    R[t]->depth = D;
    R[t]->tested.assign(D + 1, 0);
    R[t]->kept.assign(D + 1, 0);
    R[t]->nodes.assign((size_t)(D + 1) * k, 0);
    R[t]->recheck.assign(D + 1, 0);
    R[t]->recheck64.assign(D + 1, 0);
    R[t]->madds.assign(D + 1, 0);
    // an empty tree until the system finishes (a system whose boxes all go keeps it)
    int64_t N0[VX_KMAX] = {0};
    if (csf_alloc(&R[t]->fin, k, D, N0, s) != VX_OK || set_ptr_sentinels(R[t]->fin.v, s) != VX_OK)
      rc = VX_ENOMEM;
    R[t]->fin_set = true;
  }
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (rc == VX_OK && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess))
    rc = VX_ECUDA;
  int *h_status = nullptr;  // pinned: the device status word, read with a level's last wait
  if (rc == VX_OK && cudaHostAlloc((void **)&h_status, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    set_error("cudaHostAlloc of the status word failed");
    h_status = nullptr;
    rc = VX_ENOMEM;
  }
  if (rc == VX_OK && cudaEventRecord(ev0, s) != cudaSuccess) rc = VX_ECUDA;
  // level 0: one box per tree
  Forest cur;
  if (rc == VX_OK) {
    int64_t N[VX_KMAX];
    for (int d = 0; d < VX_KMAX; ++d) N[d] = S;
    rc = csf_alloc(&cur.c, k, 0, N, s);
    if (rc == VX_OK) {
      k_forest_level0<<<grid1(S + 1), 256, 0, s>>>(cur.c.v, S);
      note_launch();
      cur.off.assign((size_t)k * (S + 1), 0);
      for (int d = 0; d < k; ++d)
        for (int t = 0; t <= S; ++t) cur.off[(size_t)d * (S + 1) + t] = t;
      rc = upload_off(cur, k, S, s);
    }
  }
  std::vector<int64_t> hseg;
  for (int l = 0; l <= maxdepth && rc == VX_OK; ++l) {
    const int64_t n = cur.c.v.N[k - 1];
    bool any_final = false, any_cont = false;
    for (int t = 0; t < S; ++t) {
      if (tdep[t] < l) continue;
      const int64_t nt = cur.off[(size_t)(k - 1) * (S + 1) + t + 1] - cur.off[(size_t)(k - 1) * (S + 1) + t];
      R[t]->tested[l] = nt;
      for (int d = 0; d < k; ++d)
        R[t]->nodes[(size_t)l * k + d] =
            cur.off[(size_t)d * (S + 1) + t + 1] - cur.off[(size_t)d * (S + 1) + t];
      if (nt > 0) (tdep[t] == l ? any_final : any_cont) = true;
      LevelGrid g;
      rc = make_grid(k, domains + doff[ids[t]], l, &g);
      if (rc != VX_OK) break;
      for (int d = 0; d < k; ++d) ht[t].ax[d] = g.ax[d];
    }
    if (rc != VX_OK || n == 0) break;
    rc = l == 0 ? dmalloc_copy_trees(d_trees, ht, s) : copy_tree_grids(d_trees, d_ax, ht, s);
    uint8_t *keep = nullptr, *flag = nullptr, *m = nullptr;
    if (rc == VX_OK) rc = dmalloc((void **)&keep, (size_t)n, s);
    if (rc == VX_OK) rc = dmalloc((void **)&flag, (size_t)n, s);
    if (rc == VX_OK) rc = dmalloc((void **)&m, (size_t)n, s);
    // evaluate: the arithmetic of opts; binary64 for the flagged boxes (VX_FP32: the error
    // band; VX_FP32_MIDRAD: tight boxes with fp64_recheck, every box of a finishing tree with
    // fp64_final)
    const int arith = opts.mode == VX_FP64 ? ARITH_F64
                      : (opts.mode == VX_FP32 ? ARITH_F32_CERT : ARITH_F32_MIDRAD);
    const bool flagged = opts.mode == VX_FP32 || (opts.mode == VX_FP32_MIDRAD && opts.fp64_recheck);
    int64_t w = 0;
    if (rc == VX_OK)
      rc = eval_forest(arith, d_trees, ht.data(), cur.d_off, cur.off.data(), S, cur.c.v, keep,
                       flagged ? flag : nullptr, theta, s, &w);
    if (rc == VX_OK && !flagged && (opts.mode == VX_FP32_MIDRAD && opts.fp64_final))
      if (cudaMemsetAsync(flag, 0, (size_t)n, s) != cudaSuccess) rc = VX_ECUDA;
    const bool defer = opts.mode == VX_FP32 && opts.recheck_last != 0;
    const bool recheck = (flagged && (!defer || any_final)) ||
                         (opts.mode == VX_FP32_MIDRAD && opts.fp64_final && any_final);
    if (rc == VX_OK && defer && any_final) {
      k_tree_mask<<<grid1((n + 15) / 16), 256, 0, s>>>(keep, cur.d_off + (int64_t)(k - 1) * (S + 1), S,
                                           d_tdep, l, 3, n, flag);
      note_launch();
    }
    if (rc == VX_OK && opts.mode == VX_FP32_MIDRAD && opts.fp64_final && any_final) {
      k_tree_mask<<<grid1((n + 15) / 16), 256, 0, s>>>(keep, cur.d_off + (int64_t)(k - 1) * (S + 1), S,
                                           d_tdep, l, 2, n, flag);
      note_launch();
    }
    // per-tree madds of the level (host, from the counts)
    for (int t = 0; t < S && rc == VX_OK; ++t) {
      if (tdep[t] < l) continue;
      int64_t mt = 0;
      for (int f = 0; f < ht[t].dev.npoly; ++f)
        for (int d = 0; d < k; ++d) {
          const StageDev &st = ht[t].dev.p[f].st[d];
          mt += (cur.off[(size_t)d * (S + 1) + t + 1] - cur.off[(size_t)d * (S + 1) + t]) *
                (st.blk_in - st.nfib);
        }
      R[t]->madds[l] += mt;
    }
    if (rc == VX_OK && recheck) {
      // the flagged leaves as a forest of their own, in binary64; decisions scattered back
      Forest sub;
      int32_t *idx = nullptr;
      uint8_t *subkeep = nullptr;
      rc = dmalloc((void **)&idx, (size_t)n * sizeof(int32_t), s);
      if (rc == VX_OK) rc = prune_forest(cur, flag, 0, idx, k, S, d_seg, hseg, s, sub);
      const int64_t ns = sub.c.v.N[k - 1];
      for (int t = 0; t < S && rc == VX_OK; ++t)
        if (tdep[t] >= l) {
          R[t]->recheck[l] = sub.off[(size_t)(k - 1) * (S + 1) + t + 1] -
                             sub.off[(size_t)(k - 1) * (S + 1) + t];
          R[t]->recheck64[l] = R[t]->recheck[l];
        }
      if (rc == VX_OK && ns > 0) {
        rc = dmalloc((void **)&subkeep, (size_t)ns, s);
        int64_t w2 = 0;
        if (rc == VX_OK)
          rc = eval_forest(ARITH_F64, d_trees, ht.data(), sub.d_off, sub.off.data(), S, sub.c.v,
                           subkeep, nullptr, 0.f, s, &w2);
        if (rc == VX_OK) rc = scatter_keep(idx, subkeep, ns, keep, s);
      }
      dfree(subkeep, s);
      dfree(idx, s);
      release(sub, s);
    }
    // finishing trees: their kept boxes are the result, each tree's as a CSF of its own
    if (rc == VX_OK && any_final) {
      Forest fin;
      k_tree_mask<<<grid1((n + 15) / 16), 256, 0, s>>>(keep, cur.d_off + (int64_t)(k - 1) * (S + 1), S,
                                           d_tdep, l, 0, n, m);
      note_launch();
      rc = prune_forest(cur, m, 0, nullptr, k, S, d_seg, hseg, s, fin);
      for (int t = 0; t < S && rc == VX_OK; ++t) {
        if (tdep[t] != l) continue;
        TreeSlice ts;
        int64_t N[VX_KMAX] = {0};
        for (int d = 0; d < VX_KMAX; ++d) ts.o[d] = ts.n[d] = 0;
        for (int d = 0; d < k; ++d) {
          ts.o[d] = fin.off[(size_t)d * (S + 1) + t];
          ts.n[d] = N[d] = fin.off[(size_t)d * (S + 1) + t + 1] - ts.o[d];
        }
        R[t]->kept[l] = N[k - 1];
        csf_release(&R[t]->fin);
        rc = csf_alloc(&R[t]->fin, k, l, N, s);
        if (rc == VX_OK) {
          k_tree_extract<<<grid1(N[k - 1] + 1), 256, 0, s>>>(fin.c.v, ts, R[t]->fin.v);
          note_launch();
          if (cudaGetLastError() != cudaSuccess) rc = VX_ECUDA;
        }
      }
      release(fin, s);
    }
    // the others go on: bisect their kept boxes into the next level's forest
    Forest next;
    if (rc == VX_OK) {
      k_tree_mask<<<grid1((n + 15) / 16), 256, 0, s>>>(keep, cur.d_off + (int64_t)(k - 1) * (S + 1), S,
                                           d_tdep, l, 1, n, m);
      note_launch();
      if (any_cont) {
        // the level's device status travels back in the prune's wait (every kernel that
        // can give up a bounded wait ran before it)
        *h_status = 0;
        rc = queue_device_status(s, h_status);
        if (rc == VX_OK) rc = prune_forest(cur, m, 1, nullptr, k, S, d_seg, hseg, s, next);
        for (int t = 0; t < S && rc == VX_OK; ++t)
          if (tdep[t] > l)
            R[t]->kept[l] = hseg[(size_t)(k - 1) * (S + 1) + t + 1] - hseg[(size_t)(k - 1) * (S + 1) + t];
      }
    }
    dfree(m, s);
    dfree(flag, s);
    dfree(keep, s);
    int st = 0;
    if (rc == VX_OK) {
      if (any_cont && *h_status == 0)
        st = 0;  // read in the prune's wait
      else
        rc = take_device_status(s, &st);  // waits; clears a set status
    }
    if (rc == VX_OK && st) {
      set_error("a bounded device wait gave up at level %d", l);
      rc = VX_ETIMEOUT;
    }
    release(cur, s);
    if (rc != VX_OK || !any_cont) {
      release(next, s);
      break;
    }
    cur = next;
  }
  release(cur, s);
  if (rc == VX_OK) {
    float ms = 0.f;
    cudaError_t e = cudaEventRecord(ev1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
    if (e != cudaSuccess) {
      set_error("batch: %s", cudaGetErrorString(e));
      rc = VX_ECUDA;
    }
    for (int t = 0; t < S; ++t) R[t]->elapsed_ms = ms;  // the group's wall time
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  dfree(d_seg, s);
  dfree(d_tdep, s);
  dfree(d_ax, s);
  dfree(d_trees, s);
  if (cudaStreamSynchronize(s) != cudaSuccess && rc == VX_OK) rc = VX_ECUDA;
  if (h_status) cudaFreeHost(h_status);
  if (rc == VX_OK) {  // a status that no level's wait carried back (an empty last prune)
    int st = 0;
    rc = take_device_status(s, &st);
    if (rc == VX_OK && st) {
      set_error("a bounded device wait gave up");
      rc = VX_ETIMEOUT;
    }
  }
  for (int t = 0; t < S; ++t) vx_system_free(sysv[t]);
  for (int t = 0; t < S; ++t) {
    if (rc == VX_OK)
      out[ids[t]] = R[t];
    else
      vx_result_free(R[t]);
  }
  return rc;
}

}  // namespace
}  // namespace vx

int vx_enclose_batch(const vx_poly *const *systems, const int32_t *npoly, const double *domains,
                     const int32_t *depths, int32_t nsys, const vx_opts *opts, int32_t nworkers,
                     vx_result **out) {
  clear_error();
  (void)nworkers;
  if (!systems || !npoly || !domains || !depths || !out || nsys < 0) {
    set_error("vx_enclose_batch: NULL argument or negative count");
    return VX_EINVAL;
  }
  for (int32_t i = 0; i < nsys; ++i) out[i] = nullptr;
  if (nsys == 0) return VX_OK;
  vx_opts o{};
  if (opts) o = *opts;
  if (o.mode != VX_FP64 && o.mode != VX_FP32_MIDRAD && o.mode != VX_FP32) {
    set_error("vx_enclose_batch: unknown mode %d", o.mode);
    return VX_EINVAL;
  }
  if (o.taylor_order != 0) {
    set_error("vx_enclose_batch: the Taylor form is not available in batches");
    return VX_EINVAL;
  }
  if (o.recheck_last != 0 && o.mode != VX_FP32) {
    set_error("vx_enclose_batch: recheck_last needs VX_FP32");
    return VX_EINVAL;
  }
  // domain offsets: system i owns 2 * k_i doubles; groups of equal k
  std::vector<int64_t> doff(nsys + 1, 0);
  std::vector<std::vector<int32_t>> groups(VX_KMAX + 1);
  for (int32_t i = 0; i < nsys; ++i) {
    if (!systems[i] || npoly[i] < 1) {
      set_error("vx_enclose_batch: system %d has no polynomials", i);
      return VX_EINVAL;
    }
    const int k = systems[i][0].nvars;
    if (k < 1 || k > VX_KMAX) {
      set_error("vx_enclose_batch: system %d has %d variables (1..%d)", i, k, VX_KMAX);
      return VX_EINVAL;
    }
    doff[i + 1] = doff[i] + 2 * (int64_t)k;
    groups[k].push_back(i);
  }
  cudaStream_t s = library_stream();
  int rc = VX_OK;
  for (int k = 1; k <= VX_KMAX && rc == VX_OK; ++k)
    if (!groups[k].empty()) rc = batch_group(groups[k], systems, npoly, domains, doff, depths, o, s, out);
  if (rc != VX_OK) {
    const std::string msg = std::string("vx_enclose_batch: ") + vx_last_error();
    for (int32_t i = 0; i < nsys; ++i) {
      vx_result_free(out[i]);
      out[i] = nullptr;
    }
    set_error("%s", msg.c_str());
  }
  return rc;
}

int vx_result_boxes(vx_result *R, int64_t *n, const int32_t **h_tuples) {
  clear_error();
  if (!R || !n || !h_tuples) {
    set_error("vx_result_boxes: NULL argument");
    return VX_EINVAL;
  }
  if (R->hcount < 0) {
    const int k = R->k;
    const auto trees = result_trees(R);
    int64_t m = 0, mmax = 0;
    for (auto *t : trees) {
      m += t->v.N[k - 1];
      mmax = std::max<int64_t>(mmax, t->v.N[k - 1]);
    }
    if (m > 0) {
      cudaStream_t s = R->fin.stream;
      void *hb = nullptr;
      size_t cap = 0;
      VX_CHECK(pinned_get((size_t)m * k * 4, &hb, &cap));
      int32_t *d = nullptr;
      int rc = dmalloc((void **)&d, (size_t)mmax * k * 4, s);
      int64_t at = 0;
      for (size_t j = 0; j < trees.size() && rc == VX_OK; ++j) {
        const int64_t mj = trees[j]->v.N[k - 1];
        if (mj == 0) continue;
        rc = csf_tuples_dev(trees[j]->v, d, s);
        if (rc == VX_OK) {
          cudaError_t e = cudaMemcpyAsync((int32_t *)hb + at * k, d, (size_t)mj * k * 4,
                                          cudaMemcpyDeviceToHost, s);
          if (e == cudaSuccess) e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) {
            set_error("copying the boxes to the host failed: %s", cudaGetErrorString(e));
            rc = VX_ECUDA;
          }
        }
        at += mj;
      }
      dfree(d, s);
      if (rc != VX_OK) {
        pinned_put(hb, cap);
        return rc;
      }
      R->htup = (int32_t *)hb;
      R->hcap = cap;
    }
    R->hcount = m;
  }
  *n = R->hcount;
  *h_tuples = R->htup;
  return VX_OK;
}

int vx_result_box_codes(vx_result *R, int64_t *n, int32_t *code_bytes, const void **h_codes) {
  clear_error();
  if (!R || !n || !code_bytes || !h_codes) {
    set_error("vx_result_box_codes: NULL argument");
    return VX_EINVAL;
  }
  const int k = R->k;
  const int cb = k * R->depth <= 32 ? 4 : 8;
  if (R->hcodes_count < 0) {
    const auto trees = result_trees(R);
    int64_t m = 0, mmax = 0;
    for (auto *t : trees) {
      m += t->v.N[k - 1];
      mmax = std::max<int64_t>(mmax, t->v.N[k - 1]);
    }
    if (m > 0) {
      cudaStream_t s = R->fin.stream;
      void *hb = nullptr;
      size_t cap = 0;
      VX_CHECK(pinned_get((size_t)m * cb, &hb, &cap));
      // the codes kernel writes straight into the pinned buffer when the device can address
      // it (a mapped allocation: the stores cross the host link as they are made), else into
      // device memory followed by a copy
      void *dh = nullptr;
      int rc = VX_OK;
      if (kCodesToHost && cudaHostGetDevicePointer(&dh, hb, 0) == cudaSuccess && dh) {
        int64_t at = 0;
        for (size_t j = 0; j < trees.size() && rc == VX_OK; ++j) {
          const int64_t mj = trees[j]->v.N[k - 1];
          if (mj == 0) continue;
          rc = csf_box_codes_dev(trees[j]->v, (char *)dh + (size_t)at * cb, s);
          at += mj;
        }
        if (rc == VX_OK && cudaStreamSynchronize(s) != cudaSuccess) {
          set_error("writing the box codes to the host failed: %s",
                    cudaGetErrorString(cudaGetLastError()));
          rc = VX_ECUDA;
        }
        if (rc != VX_OK) {
          pinned_put(hb, cap);
          return rc;
        }
        R->hcodes = hb;
        R->hcodes_cap = cap;
        R->hcodes_count = m;
        *n = R->hcodes_count;
        *code_bytes = cb;
        *h_codes = R->hcodes;
        return VX_OK;
      }
      cudaGetLastError();  // a buffer the device cannot address: the copy below
      void *d = nullptr;
      rc = dmalloc(&d, (size_t)mmax * cb, s);
      int64_t at = 0;
      for (size_t j = 0; j < trees.size() && rc == VX_OK; ++j) {
        const int64_t mj = trees[j]->v.N[k - 1];
        if (mj == 0) continue;
        rc = csf_box_codes_dev(trees[j]->v, d, s);
        if (rc == VX_OK) {
          cudaError_t e = cudaMemcpyAsync((char *)hb + (size_t)at * cb, d, (size_t)mj * cb,
                                          cudaMemcpyDeviceToHost, s);
          if (e == cudaSuccess) e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) {
            set_error("copying the box codes to the host failed: %s", cudaGetErrorString(e));
            rc = VX_ECUDA;
          }
        }
        at += mj;
      }
      dfree(d, s);
      if (rc != VX_OK) {
        pinned_put(hb, cap);
        return rc;
      }
      R->hcodes = hb;
      R->hcodes_cap = cap;
    }
    R->hcodes_count = m;
  }
  *n = R->hcodes_count;
  *code_bytes = cb;
  *h_codes = R->hcodes;
  return VX_OK;
}

int vx_result_included(vx_result *R, int64_t *n, const int32_t **h_levels,
                       const int32_t **h_tuples) {
  clear_error();
  if (!R || !n || !h_levels || !h_tuples) {
    set_error("vx_result_included: NULL argument");
    return VX_EINVAL;
  }
  if (R->hinc_count < 0) {
    const int k = R->k;
    int64_t total = 0;
    for (auto &lc : R->incl) total += lc.second.v.N[k - 1];
    try {
      R->hinc_lev.resize((size_t)std::max<int64_t>(total, 1));
      R->hinc_tup.resize((size_t)std::max<int64_t>(total, 1) * k);
    } catch (...) {
      set_error("vx_result_included: out of host memory");
      return VX_ENOMEM;
    }
    int64_t at = 0;
    for (auto &lc : R->incl) {
      const int64_t m = lc.second.v.N[k - 1];
      if (m == 0) continue;
      cudaStream_t s = lc.second.stream;
      int32_t *d = nullptr;
      int rc = dmalloc((void **)&d, (size_t)m * k * 4, s);
      if (rc == VX_OK) rc = csf_tuples_dev(lc.second.v, d, s);
      if (rc == VX_OK) {
        cudaError_t e = cudaMemcpyAsync(R->hinc_tup.data() + at * k, d, (size_t)m * k * 4,
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
          set_error("copying the certified boxes to the host failed: %s", cudaGetErrorString(e));
          rc = VX_ECUDA;
        }
      }
      dfree(d, s);
      VX_CHECK(rc);
      for (int64_t i = 0; i < m; ++i) R->hinc_lev[at + i] = lc.first;
      at += m;
    }
    R->hinc_count = total;
  }
  *n = R->hinc_count;
  *h_levels = R->hinc_lev.data();
  *h_tuples = R->hinc_tup.data();
  return VX_OK;
}

int vx_result_csf(const vx_result *R, const vx_csf **csf) {
  clear_error();
  if (!R || !csf) {
    set_error("vx_result_csf: NULL argument");
    return VX_EINVAL;
  }
  // vx_csf is a thin wrapper over CsfObj with the same layout
  if (R->more.empty()) {
    *csf = reinterpret_cast<const vx_csf *>(&R->fin);
    return VX_OK;
  }
  // an enclosure run in x_1 ranges: one tree of all its boxes, made once
  vx_result *W = const_cast<vx_result *>(R);
  if (!W->merged_set) {
    const int k = R->k;
    const auto trees = result_trees(R);
    int64_t m = 0;
    for (auto *t : trees) m += t->v.N[k - 1];
    if (m > INT32_MAX) {
      set_error("vx_result_csf: %lld boxes exceed one tree's 32-bit indices (use "
                "vx_result_boxes or vx_result_box_codes)", (long long)m);
      return VX_EOVERFLOW;
    }
    cudaStream_t s = R->fin.stream;
    int32_t *d = nullptr;
    VX_CHECK(dmalloc((void **)&d, (size_t)std::max<int64_t>(m, 1) * k * 4, s));
    int rc = VX_OK;
    int64_t at = 0;
    for (size_t j = 0; j < trees.size() && rc == VX_OK; ++j) {
      rc = csf_tuples_dev(trees[j]->v, d + at * k, s);
      at += trees[j]->v.N[k - 1];
    }
    if (rc == VX_OK) rc = csf_build_dev(k, R->depth, d, m, s, &W->merged, nullptr);
    dfree(d, s);
    VX_CHECK(rc);
    W->merged_set = true;
  }
  *csf = reinterpret_cast<const vx_csf *>(&R->merged);
  return VX_OK;
}

int vx_result_stats(const vx_result *R, int32_t *nlevels, int64_t *tested, int64_t *kept,
                    int64_t *nodes, int64_t *recheck, int64_t *madds) {
  clear_error();
  if (!R) {
    set_error("vx_result_stats: NULL result");
    return VX_EINVAL;
  }
  const int L = R->depth + 1;
  if (nlevels) *nlevels = L;
  if (tested) std::memcpy(tested, R->tested.data(), L * 8);
  if (kept) std::memcpy(kept, R->kept.data(), L * 8);
  if (nodes) std::memcpy(nodes, R->nodes.data(), (size_t)L * R->k * 8);
  if (recheck) std::memcpy(recheck, R->recheck.data(), L * 8);
  if (madds) std::memcpy(madds, R->madds.data(), L * 8);
  return VX_OK;
}

int vx_result_recheck64(const vx_result *R, int64_t *per_level) {
  clear_error();
  if (!R || !per_level) {
    set_error("vx_result_recheck64: NULL argument");
    return VX_EINVAL;
  }
  std::memcpy(per_level, R->recheck64.data(), (size_t)(R->depth + 1) * 8);
  return VX_OK;
}

int vx_result_timing(const vx_result *R, int32_t *nkinds, double *h_ms, int64_t *h_launches,
                     int64_t *h_work) {
  clear_error();
  if (!R) {
    set_error("vx_result_timing: NULL result");
    return VX_EINVAL;
  }
  if (nkinds) *nkinds = KK_COUNT;
  for (int i = 0; i < KK_COUNT; ++i) {
    if (h_ms) h_ms[i] = R->tm.ms[i];
    if (h_launches) h_launches[i] = R->tm.launches[i];
    if (h_work) h_work[i] = R->tm.work[i];
  }
  return VX_OK;
}

const char *vx_kernel_kind_name(int32_t kind) {
  return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "";
}

int vx_result_elapsed_ms(const vx_result *R, double *ms) {
  clear_error();
  if (!R || !ms) {
    set_error("vx_result_elapsed_ms: NULL argument");
    return VX_EINVAL;
  }
  *ms = R->elapsed_ms;
  return VX_OK;
}

void vx_result_free(vx_result *R) {
  if (!R) return;
  pinned_put(R->htup, R->hcap);
  pinned_put(R->hcodes, R->hcodes_cap);
  result_release_trees(R);
  R->tm.release();
  delete R;
}

}  // extern "C"
