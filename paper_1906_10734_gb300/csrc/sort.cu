// Stable LSD radix sort of (u64 key, u32 value) pairs and an exclusive scan,
// the HBM-bound primitives of the tree build.
#include <atomic>

#include "hpm_internal.cuh"

namespace hpm {
namespace {


__device__ __forceinline__ int warp_incl_scan(int v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of a block's values; returns the block total.
__device__ __forceinline__ int block_excl_scan(int v, int *ex, int *sh_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int inc = warp_incl_scan(v);
  if (lane == 31) sh_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    int t = lane < nw ? sh_warp[lane] : 0;
    t = warp_incl_scan(t);
    sh_warp[lane] = t;
  }
  __syncthreads();
  int base = w > 0 ? sh_warp[w - 1] : 0;
  *ex = base + inc - v;
  int total = sh_warp[nw - 1];
  __syncthreads();
  return total;
}

// Single-pass exclusive scan with decoupled look-back. Tiles are handed out
// in the order of a ticket counter, so every tile's predecessors are running
// or finished; each tile publishes its sum at once and its inclusive prefix
// as soon as it knows it, and reads back over its predecessors' published
// values (one warp, 32 tiles per step) until it meets a prefix. A status word
// is (flag << 62) | (epoch << 32) | value with flag 1 = sum, 2 = prefix; the
// epoch tags one call, so the words never need clearing. The last tile to
// take a ticket resets the counter for the next call. Waits are bounded: a
// wait that runs out sets kErrTimeout and the tile goes on with what it has.
constexpr int kLbThreads = 256, kLbItems = 8, kLbTile = kLbThreads * kLbItems;

__device__ __forceinline__ void st_release64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kLbThreads) k_scan_lb(const int *__restrict__ in, int *__restrict__ out, int64_t n,
                                                        int *__restrict__ total, unsigned *ticket,
                                                        unsigned long long *status, unsigned epoch, int ntiles,
                                                        int *err) {
  __shared__ int sh[32];
  __shared__ int s_tile, s_prefix;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    if (t == (unsigned)ntiles - 1) atomicExch(ticket, 0u);
    s_tile = (int)t;
  }
  __syncthreads();
  const int tile = s_tile;
  const int64_t base = (int64_t)tile * kLbTile + (int64_t)threadIdx.x * kLbItems;
  int v[kLbItems];
  int sum = 0;
#pragma unroll
  for (int k = 0; k < kLbItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    sum += v[k];
  }
  int ex;
  const int agg = block_excl_scan(sum, &ex, sh);
  const unsigned long long tag = (unsigned long long)(epoch & 0x3FFFFFFFu) << 32;
  if (threadIdx.x < 32) {
    int prefix = 0;
    if (tile == 0) {
      if (lane == 0) st_release64(status, (2ull << 62) | tag | (unsigned)agg);
    } else {
      if (lane == 0) st_release64(status + tile, (1ull << 62) | tag | (unsigned)agg);
      bool ok = true;
      for (int j = tile - 1;; j -= 32) {
        const int idx = j - lane;
        int flag = 2, val = 0;
        if (idx >= 0) {
          unsigned long long w = 0;
          for (long it = 0;; ++it) {
            w = ld_acquire64(status + idx);
            if ((w & (0x3FFFFFFFull << 32)) == tag && (w >> 62)) break;
            if (it > (1l << 22)) {
              ok = false;
              w = (2ull << 62) | tag;  // give up: take it as a zero prefix
              break;
            }
            __nanosleep(32);
          }
          flag = (int)(w >> 62);
          val = (int)(unsigned)w;
        }
        const unsigned pm = __ballot_sync(0xffffffffu, flag == 2);
        const int first = pm ? __ffs(pm) - 1 : 32;  // nearest published prefix in this window
        int add = lane <= first ? val : 0;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) add += __shfl_xor_sync(0xffffffffu, add, o);
        prefix += add;
        if (pm) break;
      }
      if (!__all_sync(0xffffffffu, ok) && lane == 0 && err) atomicOr(err, kErrTimeout);
      if (lane == 0) st_release64(status + tile, (2ull << 62) | tag | (unsigned)(prefix + agg));
    }
    if (lane == 0) s_prefix = prefix;
  }
  __syncthreads();
  int run = s_prefix + ex;
#pragma unroll
  for (int k = 0; k < kLbItems; ++k)
    if (base + k < n) {
      out[base + k] = run;
      run += v[k];
    }
  if (total && tile == ntiles - 1 && threadIdx.x == 0) *total = s_prefix + agg;
}

// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kRadix = 256;
static_assert(kSortTile == kSortTileElems && kRadix == kRadixDigits, "sort sizing shared with the static sort");

// Digits of RB bits (8 or 9: 256 or 512 counters, kDigitsPerThread per thread).
template <int RB>
struct Digits {
  static constexpr int kN = 1 << RB;
  static constexpr unsigned kMask = kN - 1;
  static constexpr int kPerThread = kN / kSortThreads;
  static_assert(kPerThread >= 1 && kN % kSortThreads == 0, "whole digits per thread");
};

template <int RB>
__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int *__restrict__ hist, int nblk) {
  using Dg = Digits<RB>;
  __shared__ int cnt[Dg::kN];
#pragma unroll
  for (int q = 0; q < Dg::kPerThread; ++q) cnt[q * kSortThreads + threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  // all of the thread's keys in flight at once, then the counts
  uint64_t k[kSortRounds];
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r) {
    const int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    k[r] = i < n ? keys[i] : 0;
  }
#pragma unroll
  for (int r = 0; r < kSortRounds; ++r)
    if (base + (int64_t)r * kSortThreads + threadIdx.x < n) atomicAdd(&cnt[(k[r] >> shift) & Dg::kMask], 1);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Dg::kPerThread; ++q) {
    const int d = q * kSortThreads + threadIdx.x;
    hist[(int64_t)d * nblk + blockIdx.x] = cnt[d];
  }
}

// Stable scatter of one tile (kSortTile consecutive elements) by the current
// digit. Each warp ranks its own 512 elements (16 rounds of 32) within
// (warp, digit) with warp-private counters, so no block barrier per round;
// the tile is then put in digit order in shared memory (order within a digit:
// warp, round, lane, i.e. the input order) and written out with consecutive
// threads on consecutive positions of each digit's run.
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kWarpRounds = kSortTile / kSortThreads;  // 16 rounds of 32 per warp
constexpr int kScatterSmem = kSortTile * (int)(sizeof(uint64_t) + sizeof(uint32_t));

template <int RB>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int shift,
    const int *__restrict__ hist, const int *__restrict__ offs, int nblk, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out) {
  using Dg = Digits<RB>;
  constexpr int P = Dg::kPerThread;
  extern __shared__ __align__(16) unsigned char sraw[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sraw);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);
  __shared__ int wcnt[kSortWarps][Dg::kN];  // per warp and digit: count, then the warp's offset in the digit
  __shared__ int dstart[Dg::kN];            // first position of each digit in the sorted tile
  __shared__ int gbase[Dg::kN];             // global position of the tile's first element of each digit
  __shared__ int wsum[kSortWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int k = 0; k < kSortWarps; ++k)
#pragma unroll
    for (int q = 0; q < P; ++q) wcnt[k][q * kSortThreads + tid] = 0;
  {
    // digit starts: exclusive scan over the digits of this tile's counts
    // (thread t holds digits P t ... P t + P - 1)
    int c[P], sum = 0;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      c[q] = hist[(int64_t)(P * tid + q) * nblk + blockIdx.x];
      sum += c[q];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int before = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) before += k < w ? wsum[k] : 0;
    int run = before + inc - sum;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      dstart[P * tid + q] = run;
      run += c[q];
      gbase[P * tid + q] = offs[(int64_t)(P * tid + q) * nblk + blockIdx.x];
    }
  }
  __syncthreads();
  // ranks within (warp, digit), warp by warp
  const unsigned lt = (1u << lane) - 1u;
  uint64_t kk[kWarpRounds];
  uint32_t vv[kWarpRounds];
  int rk[kWarpRounds];
  const int64_t wb = base + (int64_t)w * (kWarpRounds * 32);
  // the warp's keys and values in flight at once (the ranking below orders
  // its shared-memory counters with warp barriers, which loads do not cross)
#pragma unroll
  for (int r = 0; r < kWarpRounds; ++r) {
    const int64_t i = wb + r * 32 + lane;
    const bool valid = i < n;
    kk[r] = valid ? keys[i] : 0;
    vv[r] = valid ? (vals ? vals[i] : (uint32_t)i) : 0u;
  }
#pragma unroll
  for (int r = 0; r < kWarpRounds; ++r) {
    const int64_t i = wb + r * 32 + lane;
    const bool valid = i < n;
    const uint64_t key = kk[r];
    const int d = valid ? (int)((key >> shift) & Dg::kMask) : Dg::kN;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int leader = __ffs(peers) - 1, rank = __popc(peers & lt);
    int old = 0;
    if (valid && rank == 0) {
      old = wcnt[w][d];
      wcnt[w][d] = old + __popc(peers);
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    __syncwarp();
    rk[r] = old + rank;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int d = q * kSortThreads + tid;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) {
      const int c = wcnt[k][d];
      wcnt[k][d] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kWarpRounds; ++r) {
    if (wb + r * 32 + lane < n) {
      const int d = (int)((kk[r] >> shift) & Dg::kMask);
      const int pos = dstart[d] + wcnt[w][d] + rk[r];
      sk[pos] = kk[r];
      sv[pos] = vv[r];
    }
  }
  __syncthreads();
  const int nt = (int)min((int64_t)kSortTile, n - base);
  for (int j = tid; j < nt; j += kSortThreads) {
    const uint64_t key = sk[j];
    const int d = (int)((key >> shift) & Dg::kMask);
    const int p = gbase[d] + (j - dstart[d]);
    keys_out[p] = key;
    vals_out[p] = sv[j];
  }
}

}  // namespace

hpm_status exclusive_scan_i32(const int *in, int *out, int64_t n, int *d_total, const ScanCtl &ctl,
                              cudaStream_t st, int64_t *launches) {
  if (n <= 0) {
    if (d_total) HPM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), st));
    return HPM_OK;
  }
  const int64_t nt = (n + kLbTile - 1) / kLbTile;
  if (nt > ctl.tiles) return HPM_ERR_INVALID_ARG;
  static std::atomic<unsigned> epoch{1};
  k_scan_lb<<<(unsigned)nt, kLbThreads, 0, st>>>(in, out, n, d_total, ctl.ticket, ctl.status,
                                                  epoch.fetch_add(1u), (int)nt, ctl.err);
  HPM_LAUNCHED(launches);
  return HPM_OK;
}

static_assert(kLbTile == kScanTileElems, "scan sizing shared with the static sort");
int64_t scan_tiles(int64_t n) { return scan_tiles_of(n); }

// Control words of the scan in a buffer of its own, zeroed when it grows.
hpm_status ensure_scan_ctl(DevBuf &buf, int64_t tiles, int *err, cudaStream_t st, ScanCtl *out) {
  const size_t bytes = 256 + sizeof(unsigned long long) * (size_t)(tiles > 0 ? tiles : 1);
  if (bytes > buf.cap || !buf.p) {
    HPM_TRY(buf.ensure(bytes, st));
    HPM_CUDA(cudaMemsetAsync(buf.p, 0, buf.cap, st));
  }
  out->ticket = buf.as<unsigned>();
  out->status = reinterpret_cast<unsigned long long *>(buf.as<unsigned char>() + 256);
  out->tiles = (int64_t)((buf.cap - 256) / sizeof(unsigned long long));
  out->err = err;
  return HPM_OK;
}

// Sorts by the low `bits` bits of the keys, stably, in passes of 8-bit
// digits, or of 9-bit digits where that takes fewer passes and wide_digits is
// set (the scratch then holds 512 counters per tile instead of 256). On
// return keys/vals point at the sorted arrays (the pointers may have been
// swapped with the *_alt buffers). vals may be null on entry: the original
// index is used then (the first pass writes it).
template <int RB>
static hpm_status sort_passes(uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals, uint32_t *&vals_alt,
                              int64_t n, int bits, DevBuf &scratch, const ScanCtl &ctl, cudaStream_t st,
                              int64_t *launches) {
  const int nblk = (int)((n + kSortTile - 1) / kSortTile);
  const int64_t hn = (int64_t)Digits<RB>::kN * nblk;
  HPM_TRY(scratch.ensure(sizeof(int) * 2 * hn, st));
  int *hist = scratch.as<int>();
  int *offs = hist + hn;
  static DeviceCache attr_cache;
  int done = 0;
  HPM_TRY(device_cached(attr_cache, [](int *v) -> hpm_status {
    HPM_CUDA(cudaFuncSetAttribute(k_radix_scatter<RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kScatterSmem));
    *v = 1;
    return HPM_OK;
  }, &done));
  bool first = true;
  for (int shift = 0; shift < bits || first; shift += RB) {
    k_radix_hist<RB><<<nblk, kSortThreads, 0, st>>>(keys, n, shift, hist, nblk);
    HPM_LAUNCHED(launches);
    HPM_TRY(exclusive_scan_i32(hist, offs, hn, nullptr, ctl, st, launches));
    k_radix_scatter<RB><<<nblk, kSortThreads, kScatterSmem, st>>>(keys, first ? nullptr : vals, n, shift, hist,
                                                                   offs, nblk, keys_alt, vals_alt);
    HPM_LAUNCHED(launches);
    uint64_t *tk = keys;
    keys = keys_alt;
    keys_alt = tk;
    uint32_t *tv = vals;
    vals = vals_alt;
    vals_alt = tv;
    first = false;
  }
  return HPM_OK;
}

hpm_status radix_sort_pairs(uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals, uint32_t *&vals_alt, int64_t n,
                            int bits, DevBuf &scratch, const ScanCtl &ctl, cudaStream_t st, int64_t *launches,
                            bool wide_digits) {
  if (n <= 0) return HPM_OK;
  if (wide_digits && (bits + 8) / 9 < (bits + 7) / 8)
    return sort_passes<9>(keys, keys_alt, vals, vals_alt, n, bits, scratch, ctl, st, launches);
  return sort_passes<8>(keys, keys_alt, vals, vals_alt, n, bits, scratch, ctl, st, launches);
}

}  // namespace hpm
