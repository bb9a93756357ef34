// Stable LSD radix sort of (u64 key, u32 value) pairs and an exclusive scan,
// the HBM-bound primitives of the tree build.
#include "hpm_internal.cuh"

namespace hpm {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

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

__global__ void k_scan_reduce(const int *__restrict__ in, int64_t n, int *__restrict__ sums) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
    if (i < n) s += in[i];
  }
  int ex;
  int tot = block_excl_scan(s, &ex, sh);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums in place; writes the total.
__global__ void k_scan_sums(int *__restrict__ sums, int64_t nb, int *__restrict__ total) {
  __shared__ int sh[32];
  int run = 0;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    int64_t i = c + threadIdx.x;
    int v = i < nb ? sums[i] : 0;
    int ex;
    int tot = block_excl_scan(v, &ex, sh);
    if (i < nb) sums[i] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0 && total) *total = run;
}

__global__ void k_scan_apply(const int *__restrict__ in, int *__restrict__ out, int64_t n,
                             const int *__restrict__ sums) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  int ex;
  block_excl_scan(s, &ex, sh);
  int run = sums[blockIdx.x] + ex;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kRadix = 256;

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t n, int shift,
                             int *__restrict__ hist, int nblk) {
  __shared__ int cnt[kRadix];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int r = 0; r < kSortRounds; ++r) {
    int64_t i = base + (int64_t)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile (kSortTile consecutive elements) by the current
// 8-bit digit. Each warp ranks its own 512 elements (16 rounds of 32) within
// (warp, digit) with warp-private counters, so no block barrier per round;
// the tile is then put in digit order in shared memory (order within a digit:
// warp, round, lane, i.e. the input order) and written out with consecutive
// threads on consecutive positions of each digit's run.
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kWarpRounds = kSortTile / kSortThreads;  // 16 rounds of 32 per warp
constexpr int kScatterSmem = kSortTile * (int)(sizeof(uint64_t) + sizeof(uint32_t));

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals, int64_t n, int shift,
    const int *__restrict__ hist, const int *__restrict__ offs, int nblk, uint64_t *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out) {
  extern __shared__ __align__(16) unsigned char sraw[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sraw);
  uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kSortTile);
  __shared__ int wcnt[kSortWarps][kRadix];  // per warp and digit: count, then the warp's offset in the digit
  __shared__ int dstart[kRadix];            // first position of each digit in the sorted tile
  __shared__ int gbase[kRadix];             // global position of the tile's first element of each digit
  __shared__ int wsum[kSortWarps];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int k = 0; k < kSortWarps; ++k) wcnt[k][tid] = 0;
  {
    // digit starts: exclusive scan over the digits of this tile's counts
    const int c = hist[(int64_t)tid * nblk + blockIdx.x];
    int inc = c;
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
    dstart[tid] = before + inc - c;
    gbase[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
  }
  __syncthreads();
  // ranks within (warp, digit), warp by warp
  const unsigned lt = (1u << lane) - 1u;
  uint64_t kk[kWarpRounds];
  uint32_t vv[kWarpRounds];
  int rk[kWarpRounds];
  const int64_t wb = base + (int64_t)w * (kWarpRounds * 32);
#pragma unroll
  for (int r = 0; r < kWarpRounds; ++r) {
    const int64_t i = wb + r * 32 + lane;
    const bool valid = i < n;
    const uint64_t key = valid ? keys[i] : 0;
    const int d = valid ? (int)((key >> shift) & 0xff) : kRadix;
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
    kk[r] = key;
    vv[r] = valid ? (vals ? vals[i] : (uint32_t)i) : 0u;
  }
  __syncthreads();
  {
    int s = 0;
#pragma unroll
    for (int k = 0; k < kSortWarps; ++k) {
      const int c = wcnt[k][tid];
      wcnt[k][tid] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kWarpRounds; ++r) {
    if (wb + r * 32 + lane < n) {
      const int d = (int)((kk[r] >> shift) & 0xff);
      const int pos = dstart[d] + wcnt[w][d] + rk[r];
      sk[pos] = kk[r];
      sv[pos] = vv[r];
    }
  }
  __syncthreads();
  const int nt = (int)min((int64_t)kSortTile, n - base);
  for (int j = tid; j < nt; j += kSortThreads) {
    const uint64_t key = sk[j];
    const int d = (int)((key >> shift) & 0xff);
    const int p = gbase[d] + (j - dstart[d]);
    keys_out[p] = key;
    vals_out[p] = sv[j];
  }
}

}  // namespace

hpm_status exclusive_scan_i32(const int *in, int *out, int64_t n, int *d_total, DevBuf &scratch,
                              cudaStream_t st, int64_t *launches) {
  if (n <= 0) {
    if (d_total) HPM_CUDA(cudaMemsetAsync(d_total, 0, sizeof(int), st));
    return HPM_OK;
  }
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  HPM_TRY(scratch.ensure(sizeof(int) * nb, st));
  int *sums = scratch.as<int>();
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
  HPM_LAUNCHED(launches);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, nb, d_total);
  HPM_LAUNCHED(launches);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, n, sums);
  HPM_LAUNCHED(launches);
  return HPM_OK;
}

// Sorts by the low `bits` bits of the keys, stably. On return keys/vals point
// at the sorted arrays (the pointers may have been swapped with the *_alt
// buffers). vals may be null on entry: the original index is used then (the
// first pass writes it).
hpm_status radix_sort_pairs(uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                            uint32_t *&vals_alt, int64_t n, int bits, DevBuf &scratch,
                            cudaStream_t st, int64_t *launches) {
  if (n <= 0) return HPM_OK;
  const int nblk = (int)((n + kSortTile - 1) / kSortTile);
  const int64_t hn = (int64_t)kRadix * nblk;
  const int64_t scan_nb = (hn + kScanTile - 1) / kScanTile;
  HPM_TRY(scratch.ensure(sizeof(int) * (2 * hn + scan_nb + 64), st));
  int *hist = scratch.as<int>();
  int *offs = hist + hn;
  DevBuf sub;  // view into scratch for the scan's block sums
  sub.p = offs + hn;
  sub.cap = sizeof(int) * (scan_nb + 64);
  static bool attr = false;
  if (!attr) {
    HPM_CUDA(cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, kScatterSmem));
    attr = true;
  }
  bool first = true;
  for (int shift = 0; shift < bits || first; shift += 8) {
    k_radix_hist<<<nblk, kSortThreads, 0, st>>>(keys, n, shift, hist, nblk);
    HPM_LAUNCHED(launches);
    HPM_TRY(exclusive_scan_i32(hist, offs, hn, nullptr, sub, st, launches));
    k_radix_scatter<<<nblk, kSortThreads, kScatterSmem, st>>>(keys, first ? nullptr : vals, n, shift, hist,
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
  sub.p = nullptr;  // not owned
  sub.cap = 0;
  return HPM_OK;
}

}  // namespace hpm
