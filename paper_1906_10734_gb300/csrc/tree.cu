// Device oct-tree build (Sec. 1): Morton keys from FP64 positions, stable
// sort, then level by level the needed boxes with their particle ranges,
// child maps and 27-neighbour tables.
//
// Adaptive zones ("virtual completion", the reading used where the paper is
// silent on non-uniform trees): at level l the sources are all nonempty
// level-l dyadic boxes. A level-l box is needed iff its parent lies in the
// 3^3 neighbourhood of an internal cell at level l-1; those boxes hold every
// interaction-zone source of the cells at level l and every near box of the
// leaves at level l. The set is closed under taking parents, so it forms a
// tree of its own and the neighbours of a cell are the children of the
// neighbours of its parent.
#include <mutex>
#include <utility>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

constexpr int kThreads = 256;

struct LevelOffsets {
  int64_t off[kMaxDepth + 3];
  int nlev;
};

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | x << 32) & 0x1f00000000ffffull;
  x = (x | x << 16) & 0x1f0000ff0000ffull;
  x = (x | x << 8) & 0x100f00f00f00f00full;
  x = (x | x << 4) & 0x10c30c30c30c30c3ull;
  x = (x | x << 2) & 0x1249249249249249ull;
  return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

// Unit coordinate v = (x - o)/S in IEEE FP64 (no contraction); outside
// [0, 1] (or NaN) is an error; 21-bit cell coordinate min(floor(v 2^21),
// 2^21 - 1); level-D key from the top D bits of each coordinate.
// Batched trees: particle i of problem p (offsets[p] <= i < offsets[p+1]) gets
// the key (p << 3 D) | morton; sorting then groups particles by problem and
// the levels of all problems are built by the same launches.
// side_exp = e when the side is the power of two 2^e, else kNoPow2. Then
// v 2^21 = (x - o) 2^(21 - e) exactly, and its floor is read from the bits of
// the one FP64 subtraction (the same integer as the IEEE evaluation, without
// its further FP64 instructions, of which this GPU issues few per cycle).
constexpr int kNoPow2 = -100000;
// kOrigin0: the domain's origin is +0 in every axis, where x - o = x exactly
// (-0 included), so the subtraction (an FP64-pipe instruction) is skipped.
template <bool kOrigin0>
__global__ void k_keys(const double *__restrict__ pos, int64_t n, double ox, double oy, double oz,
                       double side, int side_exp, unsigned long long neg_zero, int depth,
                       uint64_t *__restrict__ keys,
                       int *__restrict__ err, const int64_t *__restrict__ offsets, int nprob) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t prob = 0;
  if (nprob > 1) {
    int lo = 0, hi = nprob;  // largest p with offsets[p] <= i
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (offsets[mid] <= i) lo = mid;
      else hi = mid;
    }
    prob = (uint64_t)lo;
  }
  const double o[3] = {ox, oy, oz};
  uint32_t c[3];
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double diff = kOrigin0 ? pos[3 * i + d] : __dsub_rn(pos[3 * i + d], o[d]);
    uint32_t q = 0;
    if (side_exp != kNoPow2) {
      unsigned long long b = (unsigned long long)__double_as_longlong(diff);
      // a negative diff whose scaled value rounds to -0 (|diff| <= neg_zero) counts as 0
      if ((b >> 63) && (b & 0x7FFFFFFFFFFFFFFFull) <= neg_zero) b = 0;
      // 0 <= diff <= 2^e, as bit patterns (NaN and negative values order above)
      if (b > ((unsigned long long)(side_exp + 1023) << 52)) {
        bad = true;
      } else {
        const int E = (int)(b >> 52);  // biased exponent; diff = m 2^(max(E,1) - 1075)
        const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (E ? (1ull << 52) : 0ull);
        const int sh = 1054 + side_exp - (E ? E : 1);  // >= 31: v 2^21 = m 2^-sh
        const unsigned long long f = sh >= 64 ? 0ull : (m >> sh);
        q = f >= 2097151ull ? 2097151u : (uint32_t)f;
      }
    } else {
      double v = __ddiv_rn(diff, side);
      if (!(v >= 0.0 && v <= 1.0)) {
        bad = true;
        v = 0.0;
      }
      const double s = floor(__dmul_rn(v, 2097152.0));
      q = s >= 2097151.0 ? 2097151u : (uint32_t)s;
    }
    c[d] = q >> (kMortonBits - depth);
  }
  if (bad) atomicOr(err, kErrDomain);
  keys[i] = (prob << (3 * depth)) | spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
}

// Particle range of problem p in the sorted order (its level-0 key is p).
__global__ void k_problem_ranges(int nprob, int64_t n, const uint64_t *__restrict__ skeys, int shift,
                                 int *__restrict__ rb, int *__restrict__ cnt, int *__restrict__ off,
                                 int *__restrict__ total) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  if (nprob == 1) {
    // a single problem holds every particle (no searches: 2 x log2 n dependent
    // loads), and the root offsets need no scan
    rb[0] = 0;
    cnt[0] = n > 0 ? 1 : 0;
    off[0] = 0;
    *total = cnt[0];
    return;
  }
  int lo = 0, hi = (int)n;
  while (lo < hi) {
    const int mid = lo + ((hi - lo) >> 1);
    if ((skeys[mid] >> shift) < (uint64_t)p) lo = mid + 1;
    else hi = mid;
  }
  int e = lo, top = (int)n;
  while (e < top) {
    const int mid = e + ((top - e) >> 1);
    if ((skeys[mid] >> shift) < (uint64_t)p + 1) e = mid + 1;
    else top = mid;
  }
  rb[p] = lo;
  cnt[p] = e > lo ? 1 : 0;
}

// The root cell of every nonempty problem (level 0).
__global__ void k_roots(int nprob, int64_t n, int depth, int leaf_max, const int *__restrict__ rb,
                        const int *__restrict__ has, const int *__restrict__ slot, uint64_t *key, int *beg,
                        int *end, int *parent, uint8_t *flags, int *child, int *nb, int *counters) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob || !has[p]) return;
  const int r = slot[p];
  int e = (int)n;
  for (int q = p + 1; q < nprob; ++q)
    if (has[q]) {
      e = rb[q];
      break;
    }
  key[r] = (uint64_t)p;
  beg[r] = rb[p];
  end[r] = e;
  parent[r] = -1;
  const bool internal = depth > 0 && (e - rb[p]) > leaf_max;
  flags[r] = kReal | (internal ? kInternal : kLeaf);
  for (int k = 0; k < 8; ++k) child[(int64_t)r * 8 + k] = -1;
  for (int k = 0; k < 27; ++k) nb[(int64_t)r * 27 + k] = k == 13 ? r : -1;
  atomicAdd(&counters[0], 1);
  if (!internal) atomicAdd(&counters[32 + 0], 1);
}

// The helpers below run inside the cooperative level kernel, where the box
// arrays are written by other blocks between grid barriers: plain coherent
// loads only (no __restrict__, no read-only cache path).
// Children of expanded box q: octants with particles become the next boxes
// from cb + off[q - pb] on, with their keys, ranges, parent and flags.
__device__ void fill_children_of(int64_t q, int64_t pb, int64_t cb, int level, int depth, int leaf_max,
                                 uint8_t *flags, uint64_t *key, int *beg, int *end, int *parent, int *child,
                                 const int *bnds, const int *off, int &nreal_sum, int &nleaf_sum) {
  int bnd[9];
  const uint64_t kq = key[q];
#pragma unroll
  for (int o = 0; o < 8; ++o) bnd[o] = bnds[(q - pb) * 8 + o];
  bnd[8] = end[q];
  const bool real = flags[q] & kInternal;
  int64_t idx = cb + off[q - pb];
  int nreal = 0, nleaf = 0;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    if (bnd[o + 1] > bnd[o]) {
      child[q * 8 + o] = (int)idx;
      key[idx] = (kq << 3) | (uint64_t)o;
      beg[idx] = bnd[o];
      end[idx] = bnd[o + 1];
      parent[idx] = (int)q;
      const bool internal = real && level < depth && (bnd[o + 1] - bnd[o]) > leaf_max;
      const bool leaf = real && !internal;
      flags[idx] = (real ? kReal : 0) | (internal ? kInternal : 0) | (leaf ? kLeaf : 0);
      nreal += real;
      nleaf += leaf;
      ++idx;
    } else {
      child[q * 8 + o] = -1;
    }
  }
  nreal_sum += nreal;
  nleaf_sum += nleaf;
}

// 27-neighbour list of box i at `level` into q (-1 where absent): the
// children of its parent's neighbours (rows of nb and child at level - 1).
__device__ __forceinline__ void neighbours_of(int64_t i, int level, const uint64_t *key, const int *parent,
                                              const int *child, const int *nb, int (&q)[27]) {
  const uint64_t k0 = key[i] & ((1ull << (3 * level)) - 1ull);
  const int c[3] = {(int)compact3(k0), (int)compact3(k0 >> 1), (int)compact3(k0 >> 2)};
  const int side = 1 << level;
  const int p = parent[i];
  // the parent's neighbour holding each of the 27 boxes, then its child: two
  // rounds of independent loads (the parent's row is not written at this level)
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int n0 = c[0] + k % 3 - 1, n1 = c[1] + (k / 3) % 3 - 1, n2 = c[2] + k / 9 - 1;
    q[k] = -1;
    if (n0 >= 0 && n0 < side && n1 >= 0 && n1 < side && n2 >= 0 && n2 < side) {
      const int dp = ((n0 >> 1) - (c[0] >> 1) + 1) + 3 * ((n1 >> 1) - (c[1] >> 1) + 1) +
                     9 * ((n2 >> 1) - (c[2] >> 1) + 1);
      q[k] = nb[(int64_t)p * 27 + dp];
    }
  }
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int n0 = c[0] + k % 3 - 1, n1 = c[1] + (k / 3) % 3 - 1, n2 = c[2] + k / 9 - 1;
    q[k] = q[k] >= 0 ? child[(int64_t)q[k] * 8 + ((n0 & 1) | ((n1 & 1) << 1) | ((n2 & 1) << 2))] : -1;
  }
}

// ---------------------------------------------------------------------------
// All levels of the box tree in one cooperative launch: every block is
// resident, so the phases of a level are separated by grid-wide barriers
// instead of kernel boundaries (about 10 launches per level otherwise, most of
// them tiny at the top of the tree).
struct GridBar {
  unsigned count, gen;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier: the last block to arrive resets the count and bumps the
// generation. Bounded: a block gives up after about 2^33 cycles (a few
// seconds), or as soon as the error word shows that another block gave up;
// false then.
__device__ bool grid_sync(GridBar *gb, int *err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire(&gb->gen);
    __threadfence();
    if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
      gb->count = 0;
      __threadfence();
      atomicAdd(&gb->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(&gb->gen) == g) {
        if (*(volatile int *)err & kErrTimeout) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > (1ll << 33)) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct LevelArgs {
  int64_t *lvl;  // lvl[0], lvl[1] set on entry; lvl[2..D+1] written here
  int depth, leaf_max;
  int64_t cap;
  uint8_t *flags;
  uint64_t *key;
  int *beg, *end, *parent, *child, *nb;
  const uint64_t *skeys;
  int *bnd;   // per box of the level being split: its 8 child boundaries
  int *off;   // per box of the level being split: first child, relative to its block's
  int *bsum;  // per block: children of its boxes
  int *counters, *err;
  GridBar *gb;
};

// Marks the 27 neighbours of internal box i (its row of nb) for expansion.
__device__ __forceinline__ void mark_neighbours(const int *q, uint8_t *flags) {
  unsigned int *words = reinterpret_cast<unsigned int *>(flags);
#pragma unroll
  for (int k = 0; k < 27; ++k)
    if (q[k] >= 0) atomicOr(words + (q[k] >> 2), (unsigned int)kExpand << (8 * (q[k] & 3)));
}

// Level l (1..D) from level l - 1 = [pb, pe), whose boxes already carry their
// expansion marks:
//   1. each block takes a contiguous run of boxes: the child boundaries of
//      its boxes (one binary search per octant, four searches interleaved
//      per thread), then their child counts and block-local offsets
//   2. block offsets from the per-block totals, then the children
//   3. the neighbour tables of the new boxes; an internal one marks its 27
//      neighbours for the next level's expansion right away
// Three grid barriers per level (and one after the roots' marks); the launch
// ends at the first empty level.
constexpr int kSearchWays = 4;  // binary searches in flight per thread (8 measured slower)
__global__ void __launch_bounds__(kThreads) k_levels(LevelArgs a) {
  __shared__ int s_warp[kThreads / 32];
  __shared__ long long s_red[2][kThreads / 32];
  __shared__ int s_nb[kThreads / 32][32 * 27];  // a warp's 32 neighbour rows
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x, gtid = (int64_t)blockIdx.x * blockDim.x + tid;
  int64_t pb = a.lvl[0], pe = a.lvl[1];
  // the roots' expansion marks (a root's only neighbour is itself)
  for (int64_t i = pb + gtid; i < pe; i += gthreads)
    if (a.flags[i] & kInternal) {
      int q[27];
#pragma unroll
      for (int k = 0; k < 27; ++k) q[k] = a.nb[i * 27 + k];
      mark_neighbours(q, a.flags);
    }
  if (!grid_sync(a.gb, a.err)) return;
  for (int l = 1; l <= a.depth; ++l) {
    // 1. boundaries, counts, block-local offsets
    const int64_t m = pe - pb;
    // a level of at most one box per block (the top of the tree, where the
    // boxes are large): one box per block, one octant per warp, each warp a
    // 32-ary search (log33 of the box's particles rounds of loads instead of
    // log2); otherwise runs of boxes per block, binary searches per thread
    const bool warp_search = m <= (int64_t)gridDim.x;
    const int64_t chunk = warp_search ? 1 : ((m + gridDim.x - 1) / gridDim.x + 31) & ~int64_t(31);
    const int64_t r0 = min((int64_t)blockIdx.x * chunk, m), r1 = min(r0 + chunk, m);
    const int shift = 3 * (a.depth - l);
    {
      static_assert(kThreads / 32 == 8, "one warp per octant");
      if (warp_search && r0 < r1) {
        const int64_t i = pb + r0;
        const int oct = wid;
        int lo = a.beg[i], hi = lo;
        uint64_t kc = 0;
        if (oct > 0 && (a.flags[i] & kExpand)) {
          hi = a.end[i];
          kc = (a.key[i] << 3) | (uint64_t)oct;
        }
        // first particle of the box at or after octant `oct`: keys in [lo, hi)
        // are sorted, so the probes below kc are a prefix of the lanes
        while (hi - lo > 32) {
          const int p = lo + (int)((int64_t)(lane + 1) * (hi - lo) / 33);
          const unsigned below = __ballot_sync(0xffffffffu, (a.skeys[p] >> shift) < kc);
          const int c = __popc(below);
          const int plo = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0), phi = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
          if (c > 0) lo = plo + 1;
          if (c < 32) hi = phi;
        }
        const bool lt = lane < hi - lo && (a.skeys[lo + lane] >> shift) < kc;
        const int b0 = lo + __popc(__ballot_sync(0xffffffffu, lt));
        if (lane == 0) a.bnd[r0 * 8 + oct] = b0;
      }
      // (box, octant) items of this block: kSearchWays binary searches in lockstep per thread
      const int64_t nit = warp_search ? 0 : 8 * (r1 - r0);
      for (int64_t t0 = tid; t0 < nit; t0 += kSearchWays * kThreads) {
        int lo[kSearchWays], hi[kSearchWays];
        uint64_t kc[kSearchWays];
#pragma unroll
        for (int j = 0; j < kSearchWays; ++j) {
          const int64_t t = t0 + (int64_t)j * kThreads;
          lo[j] = 0;
          hi[j] = 0;
          kc[j] = 0;
          if (t < nit) {
            const int64_t i = pb + r0 + t / 8;
            const int oct = (int)(t & 7);
            lo[j] = a.beg[i];
            hi[j] = lo[j];
            if (oct > 0 && (a.flags[i] & kExpand)) {
              hi[j] = a.end[i];
              kc[j] = (a.key[i] << 3) | (uint64_t)oct;
            }
          }
        }
        for (;;) {
          bool any = false;
#pragma unroll
          for (int j = 0; j < kSearchWays; ++j)
            if (lo[j] < hi[j]) {
              any = true;
              const int mid = lo[j] + ((hi[j] - lo[j]) >> 1);
              if ((a.skeys[mid] >> shift) < kc[j]) lo[j] = mid + 1;
              else hi[j] = mid;
            }
          if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kSearchWays; ++j) {
          const int64_t t = t0 + (int64_t)j * kThreads;
          if (t < nit) a.bnd[r0 * 8 + t] = lo[j];
        }
      }
      __syncthreads();
      // child counts and their exclusive scan over the block's run of boxes
      int carry = 0;
      for (int64_t rb = r0; rb < r1; rb += kThreads) {
        const int64_t bi = rb + tid;
        int c = 0;
        if (bi < r1) {
          const int64_t i = pb + bi;
          if (a.flags[i] & kExpand) {
            const int *b = a.bnd + bi * 8;
            const int en = a.end[i];
#pragma unroll
            for (int o = 0; o < 8; ++o) c += (o < 7 ? b[o + 1] : en) > b[o];
          }
        }
        int inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= o) inc += v;
        }
        if (lane == 31) s_warp[wid] = inc;
        __syncthreads();
        int before = 0, round = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
          const int v = s_warp[w];
          before += w < wid ? v : 0;
          round += v;
        }
        if (bi < r1) a.off[bi] = carry + before + inc - c;
        carry += round;
        __syncthreads();
      }
      if (tid == 0) a.bsum[blockIdx.x] = carry;
    }
    if (!grid_sync(a.gb, a.err)) return;
    // 2. this block's first child and the level's total, then the children
    int64_t base, total;
    {
      long long lo = 0, all = 0;
      for (int b = tid; b < (int)gridDim.x; b += kThreads) {
        const int c = a.bsum[b];
        all += c;
        if (b < (int)blockIdx.x) lo += c;
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        lo += __shfl_xor_sync(0xffffffffu, lo, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
      }
      if (lane == 0) {
        s_red[0][wid] = lo;
        s_red[1][wid] = all;
      }
      __syncthreads();
      base = 0;
      total = 0;
#pragma unroll
      for (int w = 0; w < kThreads / 32; ++w) {
        base += s_red[0][w];
        total += s_red[1][w];
      }
      __syncthreads();
    }
    const int64_t ne = pe + total;
    if (ne > a.cap) {
      // no room for level l: the host grows the box arrays and builds again
      if (blockIdx.x == 0 && tid == 0) atomicOr(a.err, kErrCapacity);
      return;
    }
    if (blockIdx.x == 0 && tid == 0) a.lvl[l + 1] = ne;
    {
      // the level's cells and leaves, counted per warp (one atomic each, not
      // one per box on the same two words)
      int nreal = 0, nleaf = 0;
      for (int64_t bi = r0 + tid; bi < r1; bi += kThreads) {
        const int64_t q = pb + bi;
        if (!(a.flags[q] & kExpand)) {
#pragma unroll
          for (int o = 0; o < 8; ++o) a.child[q * 8 + o] = -1;
          continue;
        }
        fill_children_of(q, pb, pe + base, l, a.depth, a.leaf_max, a.flags, a.key, a.beg, a.end, a.parent,
                         a.child, a.bnd, a.off, nreal, nleaf);
      }
      nreal = __reduce_add_sync(0xffffffffu, nreal);
      nleaf = __reduce_add_sync(0xffffffffu, nleaf);
      if (lane == 0) {
        if (nreal) atomicAdd(&a.counters[l], nreal);
        if (nleaf) atomicAdd(&a.counters[32 + l], nleaf);
      }
    }
    if (total == 0) {
      // level l is empty, and so is every deeper one (every block sees the same total)
      if (blockIdx.x == 0 && tid == 0)
        for (int k = l + 2; k <= a.depth + 1; ++k) a.lvl[k] = ne;
      return;
    }
    if (!grid_sync(a.gb, a.err)) return;
    // 3. neighbour tables of level l, expansion marks for level l + 1: each
    // warp takes 32 consecutive boxes, whose rows are one contiguous run of
    // nb, staged in shared memory and written with whole-warp stores
    for (int64_t i0 = pe + gtid - lane; i0 < ne; i0 += gthreads) {
      const int64_t i = i0 + lane;
      bool real = false;
      if (i < ne) {
        const uint8_t f = a.flags[i];
        // a virtual box's row is never read (neighbour tables are read for
        // real boxes and their parents only): left unwritten
        real = f & kReal;
        if (real) {
          int q[27];
          neighbours_of(i, l, a.key, a.parent, a.child, a.nb, q);
#pragma unroll
          for (int k = 0; k < 27; ++k) s_nb[wid][lane * 27 + k] = q[k];
          if (l < a.depth && (f & kInternal)) mark_neighbours(q, a.flags);
        }
      }
      const unsigned rows = __ballot_sync(0xffffffffu, real);
      __syncwarp();
      const int cnt = (int)min((int64_t)32, ne - i0) * 27;
      for (int x = lane; x < cnt; x += 32)
        if (rows >> (x / 27) & 1u) a.nb[i0 * 27 + x] = s_nb[wid][x];
      __syncwarp();
    }
    if (!grid_sync(a.gb, a.err)) return;
    pb = pe;
    pe = ne;
  }
}

// The four work lists of a build at once (box order kept): 0 real cells at
// level >= 2 (targets), 1 leaves, 2 boxes at level >= 2 that are not
// expanded (P2G), 3 internal cells at level >= 1 (parents of targets).
// Pass 1 counts each list per block of kThreads boxes (warp ballots); one
// exclusive scan over the four lists' block counts, list after list; pass 2
// recomputes the ballots and writes every selected box at its list position.
__device__ __forceinline__ unsigned list_bits(int64_t i, int64_t nbox, int64_t off2, int64_t off1,
                                              const uint8_t *__restrict__ flags) {
  if (i >= nbox) return 0u;
  const uint8_t f = flags[i];
  return (i >= off2 && (f & kReal) ? 1u : 0u) | (f & kLeaf ? 2u : 0u) | (i >= off2 && !(f & kExpand) ? 4u : 0u) |
         (i >= off1 && (f & kInternal) ? 8u : 0u);
}

__global__ void __launch_bounds__(kThreads) k_lists_count(int64_t nbox, int64_t off2, int64_t off1,
                                                          const uint8_t *__restrict__ flags, int nblk,
                                                          int *__restrict__ cnt) {
  __shared__ int wsum[4][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned bits = list_bits((int64_t)blockIdx.x * kThreads + threadIdx.x, nbox, off2, off1, flags);
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    const int c = __popc(__ballot_sync(0xffffffffu, (bits >> L) & 1u));
    if (lane == 0) wsum[L][w] = c;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    int t = 0;
    for (int k = 0; k < kThreads / 32; ++k) t += wsum[threadIdx.x][k];
    cnt[(int64_t)threadIdx.x * nblk + blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) k_lists_write(int64_t nbox, int64_t off2, int64_t off1,
                                                          const uint8_t *__restrict__ flags, int nblk,
                                                          const int *__restrict__ off, const int *__restrict__ total,
                                                          int *__restrict__ out0, int *__restrict__ out1,
                                                          int *__restrict__ out2, int *__restrict__ out3,
                                                          int *__restrict__ totals) {
  __shared__ int wsum[4][kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const unsigned bits = list_bits(i, nbox, off2, off1, flags);
  unsigned ball[4];
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    ball[L] = __ballot_sync(0xffffffffu, (bits >> L) & 1u);
    if (lane == 0) wsum[L][w] = __popc(ball[L]);
  }
  __syncthreads();
  int *outs[4] = {out0, out1, out2, out3};
#pragma unroll
  for (int L = 0; L < 4; ++L) {
    if (!((bits >> L) & 1u)) continue;
    int before = 0;
    for (int k = 0; k < w; ++k) before += wsum[L][k];
    const int pos = off[(int64_t)L * nblk + blockIdx.x] - off[(int64_t)L * nblk] + before +
                    __popc(ball[L] & ((1u << lane) - 1u));
    outs[L][pos] = (int)i;
  }
  // each list's total: its scanned base of the next list, less its own base
  if (blockIdx.x == 0 && threadIdx.x < 4) {
    const int L = threadIdx.x;
    const int next = L < 3 ? off[(int64_t)(L + 1) * nblk] : *total;
    totals[L] = next - off[(int64_t)L * nblk];
  }
}


// Interaction zone of each target (cells at level >= 2) as its parent's 6^3
// block: box j = bx + 6 by + 36 bz is a child of the parent's neighbour
// (bx/2, by/2, bz/2); it is a source iff nonempty and at Chebyshev distance >= 2
// from the target (Sec. 1). Stored as effective-mass rows (box - off2) or -1.
__global__ void k_target_blocks(int64_t ntgt, const int *__restrict__ tgt_box, const int *__restrict__ parent,
                                const int *__restrict__ nb, const int *__restrict__ child,
                                const uint64_t *__restrict__ key, int64_t off2, LevelOffsets lo,
                                int *__restrict__ blk, int *__restrict__ info) {
  // one thread per (target, parent neighbour): the neighbour's 8 children are the
  // 2x2x2 boxes (2dx..2dx+1, 2dy.., 2dz..) of the block
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntgt * 27) return;
  const int64_t t = i / 27;
  const int k = (int)(i % 27);
  const int box = tgt_box[t];
  const int o = (int)(key[box] & 7u);
  const int tc[3] = {2 + (o & 1), 2 + ((o >> 1) & 1), 2 + ((o >> 2) & 1)};
  const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
  const int q = nb[(int64_t)parent[box] * 27 + k];
  int ch[8];
  if (q >= 0) {
    const int4 a = *reinterpret_cast<const int4 *>(child + (int64_t)q * 8);
    const int4 b = *reinterpret_cast<const int4 *>(child + (int64_t)q * 8 + 4);
    ch[0] = a.x; ch[1] = a.y; ch[2] = a.z; ch[3] = a.w; ch[4] = b.x; ch[5] = b.y; ch[6] = b.z; ch[7] = b.w;
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) ch[c] = -1;
  }
  int *out = blk + t * 216;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int bx = 2 * dx + (c & 1), by = 2 * dy + ((c >> 1) & 1), bz = 2 * dz + ((c >> 2) & 1);
    const bool far = max(abs(bx - tc[0]), max(abs(by - tc[1]), abs(bz - tc[2]))) >= 2;
    out[bx + 6 * by + 36 * bz] = (far && ch[c] >= 0) ? (int)(ch[c] - off2) : -1;
  }
  if (k == 0) {
    int l = 0;
    while (l + 1 < lo.nlev && lo.off[l + 1] <= box) ++l;
    info[t] = (l << 3) | o;
  }
}


// Leaf box of every sorted particle (a leaf's particles are contiguous).
__global__ void k_particle_box(int64_t nleaf, const int *__restrict__ leaf_box, const int *__restrict__ beg,
                               const int *__restrict__ end, int *__restrict__ pbox) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nleaf) return;
  const int box = leaf_box[l];
  for (int i = beg[box]; i < end[box]; ++i) pbox[i] = box;
}

__global__ void k_box_tgt(int64_t ntgt, const int *__restrict__ tgt_box, int *__restrict__ box_tgt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntgt) box_tgt[tgt_box[t]] = (int)t;
}

// Near-field work per leaf: nt targets times ns near sources, split into
// items of at most kP2PPairsPerItem pairs and at least kP2PMinSources sources.
// A leaf of more than kP2PSplitTargets particles is split by targets instead:
// one item per 32 targets, each against all ns sources, so no partial sums are
// stored (a source split of such a leaf would need items * nt of them).
__global__ void k_leaf_work(int64_t nleaf, const int *__restrict__ leaf_box, const int *__restrict__ nb,
                            const int *__restrict__ beg, const int *__restrict__ end, int *__restrict__ nitem,
                            int *__restrict__ part0, int *__restrict__ npart, int *__restrict__ nsrc,
                            int *__restrict__ big,
                            int *__restrict__ nbig, int *__restrict__ split, int *__restrict__ nsplit,
                            unsigned long long *__restrict__ npairs) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // near-zone pairs (i, j), j != i, of all leaves: the near field's work count
  unsigned long long pairs = 0;
  int box = -1;
  int64_t ns = 0, nt = 0;
  if (l < nleaf) {
    box = leaf_box[l];
    for (int k = 0; k < 27; ++k) {
      const int q = nb[(int64_t)box * 27 + k];
      if (q >= 0) ns += end[q] - beg[q];
    }
    nt = end[box] - beg[box];
    pairs = (unsigned long long)(nt * ns - nt);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
  if ((threadIdx.x & 31) == 0 && pairs) atomicAdd(npairs, pairs);
  // the leaf's items: a large leaf (more than kP2PSplitTargets particles) by
  // 32 targets against all sources, complete sums; else by its sources
  int64_t items = 0;
  if (l < nleaf) {
    if (nt > kP2PSplitTargets) {
      items = (nt + 31) / 32;
    } else {
      items = (nt * ns + kP2PPairsPerItem - 1) / kP2PPairsPerItem;
      const int64_t cap = (ns + kP2PMinSources - 1) / kP2PMinSources;
      if (items > cap) items = cap;
      if (items < 1) items = 1;
    }
  }
  // a split leaf's partial sums: items x nt of them, placed by an atomic
  // counter (each leaf reads back only its own), one atomic per warp; the
  // same for the lists of split leaves
  const unsigned lane = threadIdx.x & 31, lt = (1u << lane) - 1u;
  const bool by_src = l < nleaf && nt <= kP2PSplitTargets && items > 1;
  const int want = by_src ? (int)(items * nt) : 0;
  int inc = want;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  int pbase = 0;
  if (lane == 31 && inc) pbase = atomicAdd(npart, inc);
  pbase = __shfl_sync(0xffffffffu, pbase, 31);
  const bool is_big = by_src && items > kP2PCombineWarp, is_split = by_src && !is_big;
  const unsigned mb = __ballot_sync(0xffffffffu, is_big), ms = __ballot_sync(0xffffffffu, is_split);
  int bb = 0, sb = 0;
  if (lane == 0) {
    if (mb) bb = atomicAdd(nbig, __popc(mb));
    if (ms) sb = atomicAdd(nsplit, __popc(ms));
  }
  bb = __shfl_sync(0xffffffffu, bb, 0);
  sb = __shfl_sync(0xffffffffu, sb, 0);
  if (l >= nleaf) return;
  nsrc[l] = (int)ns;
  nitem[l] = (int)items;
  part0[l] = by_src ? pbase + inc - want : 0;
  if (is_big) big[bb + __popc(mb & lt)] = (int)l;
  if (is_split) split[sb + __popc(ms & lt)] = (int)l;
}

// The items of each leaf (k_leaf_work's counts and near-source totals).
__global__ void k_fill_items(int64_t nleaf, const int *__restrict__ leaf_box, const int *__restrict__ nsrc,
                             const int *__restrict__ beg, const int *__restrict__ end,
                             const int *__restrict__ nitem, const int *__restrict__ item0,
                             int *__restrict__ item_leaf, int *__restrict__ item_s0, int *__restrict__ item_s1,
                             int *__restrict__ item_t) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = l < nleaf;
  int64_t ns = 0, i0 = 0;
  int n = 0;
  bool by_targets = false;
  if (valid) {
    const int box = leaf_box[l];
    ns = nsrc[l];
    n = nitem[l];
    i0 = item0[l];
    by_targets = end[box] - beg[box] > kP2PSplitTargets;
  }
  // item k of a leaf: its targets (all, or 32 from 32 k) and its part of the
  // concatenated near sources
  auto put = [&](int64_t leaf, int64_t base, int nn, int64_t nsrc_l, bool bt, int k) {
    item_leaf[base + k] = (int)leaf;
    item_s0[base + k] = bt ? 0 : (int)(nsrc_l * k / nn);
    item_s1[base + k] = bt ? (int)nsrc_l : (int)(nsrc_l * (k + 1) / nn);
    item_t[base + k] = bt ? 32 * k : -1;
  };
  // most leaves have one item or a few; a leaf with many (a small leaf beside
  // large neighbour boxes) is written by the whole warp
  if (valid && n <= 4)
    for (int k = 0; k < n; ++k) put(l, i0, n, ns, by_targets, k);
  unsigned many = __ballot_sync(0xffffffffu, valid && n > 4);
  while (many) {
    const int src = __ffs(many) - 1;
    many &= many - 1;
    const int64_t lb = __shfl_sync(0xffffffffu, l, src), ib = __shfl_sync(0xffffffffu, i0, src),
                  nsb = __shfl_sync(0xffffffffu, ns, src);
    const int nb = __shfl_sync(0xffffffffu, n, src);
    const bool bt = __shfl_sync(0xffffffffu, by_targets, src);
    for (int k = lane; k < nb; k += 32) put(lb, ib, nb, nsb, bt, k);
  }
}

hpm_status ensure_boxes(TreeDev &t, int64_t nbox, cudaStream_t st) {
  HPM_TRY(t.box_key.ensure(sizeof(uint64_t) * nbox, st, true));
  HPM_TRY(t.box_beg.ensure(sizeof(int) * nbox, st, true));
  HPM_TRY(t.box_end.ensure(sizeof(int) * nbox, st, true));
  HPM_TRY(t.box_parent.ensure(sizeof(int) * nbox, st, true));
  HPM_TRY(t.box_flags.ensure(sizeof(uint8_t) * ((nbox + 15) & ~int64_t(15)), st, true));  // word-wide atomics in k_expand
  HPM_TRY(t.box_child.ensure(sizeof(int) * 8 * nbox, st, true));
  HPM_TRY(t.box_nb.ensure(sizeof(int) * 27 * nbox, st, true));
  return HPM_OK;
}

}  // namespace

// e if side = 2^e exactly (a normal double), else kNoPow2
static int pow2_exponent(double side) {
  int e = 0;
  const double f = std::frexp(side, &e);  // side = f 2^e, f in [0.5, 1)
  return (f == 0.5 && std::isfinite(side) && e - 1 >= -1022 && e - 1 <= 1023) ? e - 1 : kNoPow2;
}

// Bits of the largest |diff| whose product with 2^-e rounds to zero
// (2^(e - 1075), ties to even), 0 when there is none but -0.
static unsigned long long neg_zero_bits(int e) {
  if (e == kNoPow2 || e < 1) return 0ull;
  const double t = std::ldexp(1.0, e - 1075);
  unsigned long long b = 0;
  std::memcpy(&b, &t, sizeof(b));
  return b;
}

// The origin is +0 in every axis (bit patterns: -0 does not qualify).
static bool origin_is_zero(const hpm_domain &dom) {
  for (int d = 0; d < 3; ++d) {
    uint64_t b;
    memcpy(&b, &dom.origin[d], sizeof(b));
    if (b != 0) return false;
  }
  return true;
}

hpm_status launch_morton_keys(const hpm_domain &dom, int depth, const double *d_pos, int64_t n,
                              uint64_t *d_keys, int *d_err, cudaStream_t st) {
  if (n <= 0) return HPM_OK;
  (origin_is_zero(dom) ? k_keys<true> : k_keys<false>)<<<blocks_for(n), kThreads, 0, st>>>(
      d_pos, n, dom.origin[0], dom.origin[1], dom.origin[2], dom.side,
                                             pow2_exponent(dom.side), neg_zero_bits(pow2_exponent(dom.side)), depth, d_keys, d_err, nullptr, 1);
  HPM_LAUNCHED((int64_t *)nullptr);
  return HPM_OK;
}

// The plan's pinned read-back buffer (kPinBytes), allocated at its first build
// (bytes 768.. hold the solve's error word read by the host entry points).
constexpr size_t kPinBytes = 1024;
static hpm_status pinned(hpm_plan_s *pl, unsigned char **out) {
  if (!pl->h_pin) HPM_CUDA(cudaMallocHost(reinterpret_cast<void **>(&pl->h_pin), kPinBytes));
  *out = pl->h_pin;
  return HPM_OK;
}

hpm_status build_tree(hpm_plan_s *pl, const double *d_pos, int64_t n, const int64_t *h_offsets, int nprob,
                      cudaStream_t st) {
  TreeDev &t = pl->t;
  const int D = pl->max_depth;
  int64_t launches = 0;
  pl->built = false;
  pl->n = n;
  reset_work_need(pl);
  // error words: [0] this build's, [1] the solves' (kept until reported)
  const bool fresh_err = t.err.p == nullptr;
  HPM_TRY(t.err.ensure(sizeof(int) * 4, st));
  HPM_TRY(t.counters.ensure(sizeof(int) * 128, st));
  HPM_CUDA(cudaMemsetAsync(t.err.p, 0, sizeof(int) * (fresh_err ? 4 : 1), st));
  HPM_CUDA(cudaMemsetAsync(t.counters.p, 0, sizeof(int) * 128, st));
  // scans of the build: sort histograms (n / 16), problems, boxes (up to the
  // box capacity, grown below if needed), leaves
  HPM_TRY(ensure_scan_ctl(t.scan_buf, scan_tiles(std::max<int64_t>(std::max<int64_t>(n, nprob), n / 4 + 4096) + 1),
                          t.err.as<int>(), st, &t.scan));

  pl->lvl_off.assign(D + 2, 0);
  pl->depth_reached = -1;
  pl->nbox = pl->ntgt = pl->nleaf = pl->np2g = pl->ncell = 0;
  pl->nitem = pl->npart = pl->nbig = pl->nsplit = 0;
  pl->npar = 0;
  pl->tgt_lvl_off.assign(D + 2, 0);
  pl->leaf_lvl_off.assign(D + 2, 0);
  if (n == 0) {
    pl->built = true;
    pl->stats.launches = 0;
    return HPM_OK;
  }

  // keys and the stable sort by (level-D key, index)
  HPM_TRY(t.keys.ensure(sizeof(uint64_t) * n, st));
  HPM_TRY(t.keys_alt.ensure(sizeof(uint64_t) * n, st));
  HPM_TRY(t.perm.ensure(sizeof(uint32_t) * n, st));
  HPM_TRY(t.perm_alt.ensure(sizeof(uint32_t) * n, st));
  int pbits = 0;
  while ((1ll << pbits) < nprob) ++pbits;
  if (3 * D + pbits > 63) return HPM_ERR_INVALID_ARG;
  HPM_TRY(t.offsets.ensure(sizeof(int64_t) * (nprob + 1), st));
  if (nprob > 1)
    HPM_CUDA(cudaMemcpyAsync(t.offsets.p, h_offsets, sizeof(int64_t) * (nprob + 1), cudaMemcpyHostToDevice, st));
  (origin_is_zero(pl->dom) ? k_keys<true> : k_keys<false>)<<<blocks_for(n), kThreads, 0, st>>>(
      d_pos, n, pl->dom.origin[0], pl->dom.origin[1],
                                             pl->dom.origin[2], pl->dom.side, pow2_exponent(pl->dom.side),
                                             neg_zero_bits(pow2_exponent(pl->dom.side)), D,
                                             t.keys.as<uint64_t>(),
                                             t.err.as<int>(), t.offsets.as<int64_t>(), nprob);
  HPM_LAUNCHED(&launches);
  uint64_t *k0 = t.keys.as<uint64_t>(), *k1 = t.keys_alt.as<uint64_t>();
  uint32_t *v0 = t.perm.as<uint32_t>(), *v1 = t.perm_alt.as<uint32_t>();
  DevBuf &scratch = t.off;
  HPM_TRY(radix_sort_pairs(k0, k1, v0, v1, n, 3 * D + pbits, scratch, t.scan, st, &launches, true));
  // keep the sorted arrays in keys/perm
  if (k0 != t.keys.as<uint64_t>()) {
    std::swap(t.keys.p, t.keys_alt.p);
    std::swap(t.keys.cap, t.keys_alt.cap);
  }
  if (v0 != t.perm.as<uint32_t>()) {
    std::swap(t.perm.p, t.perm_alt.p);
    std::swap(t.perm.cap, t.perm_alt.cap);
  }
  const uint64_t *skeys = t.keys.as<uint64_t>();

  // level 0: the root of every nonempty problem
  HPM_TRY(t.cnt.ensure(sizeof(int) * (nprob + 1), st));
  HPM_TRY(t.off.ensure(sizeof(int) * (nprob + 1), st));
  HPM_TRY(t.bnd.ensure(sizeof(int) * (nprob + 1), st));
  k_problem_ranges<<<blocks_for(nprob), kThreads, 0, st>>>(nprob, n, skeys, 3 * D, t.bnd.as<int>(),
                                                           t.cnt.as<int>(), t.off.as<int>(),
                                                           t.counters.as<int>() + 64);
  HPM_LAUNCHED(&launches);
  if (nprob > 1)
    HPM_TRY(exclusive_scan_i32(t.cnt.as<int>(), t.off.as<int>(), nprob, t.counters.as<int>() + 64, t.scan, st,
                               &launches));
  // one problem with n > 0 particles has one root; a batch reads its count back
  unsigned char *hp = nullptr;
  HPM_TRY(pinned(pl, &hp));
  int nroot = 1;
  if (nprob > 1) {
    HPM_CUDA(cudaMemcpyAsync(hp, t.counters.as<int>() + 64, sizeof(int), cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaStreamSynchronize(st));
    memcpy(&nroot, hp, sizeof(int));
  }
  // Box capacity: grow-only across builds; the first build guesses n / 4 + 1024
  // (trees here hold 0.14-0.19 n boxes) and retries with more if it overflows.
  int64_t cap = t.box_key.cap / sizeof(uint64_t);
  cap = std::max<int64_t>(cap, std::max<int64_t>(1024 + 2 * (int64_t)nroot, n / 4 + 1024));
  HPM_TRY(ensure_boxes(t, cap, st));
  HPM_TRY(ensure_scan_ctl(t.scan_buf, scan_tiles(cap + 1), t.err.as<int>(), st, &t.scan));
  k_roots<<<blocks_for(nprob), kThreads, 0, st>>>(nprob, n, D, pl->opts.leaf_max, t.bnd.as<int>(), t.cnt.as<int>(),
                                                  t.off.as<int>(), t.box_key.as<uint64_t>(), t.box_beg.as<int>(),
                                                  t.box_end.as<int>(), t.box_parent.as<int>(),
                                                  t.box_flags.as<uint8_t>(), t.box_child.as<int>(),
                                                  t.box_nb.as<int>(), t.counters.as<int>());
  HPM_LAUNCHED(&launches);
  pl->nprob = nprob;
  HPM_TRY(t.lvl_dev.ensure(sizeof(int64_t) * (D + 2), st));
  int64_t *lvl = t.lvl_dev.as<int64_t>();
  int hc[64];
  // Levels 1..D in one cooperative launch (all blocks resident, grid-wide
  // barriers between the phases of a level); one read-back at the end.
  static DeviceCache level_cache;  // resident CTAs per SM the kernel allows
  int level_max_per_sm = 0;
  HPM_TRY(device_cached(level_cache, [](int *v) -> hpm_status {
    HPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, k_levels, kThreads, 0));
    return *v > 0 ? HPM_OK : HPM_ERR_CUDA;
  }, &level_max_per_sm));
  // CTAs per SM: the plan's tuned value (2 by default), never above what fits
  const int level_per_sm = std::min(level_max_per_sm, pl->tuning.level_blocks_per_sm > 0 ? pl->tuning.level_blocks_per_sm : 2);
  const int level_grid = level_per_sm * sm_count();
  for (int attempt = 0;; ++attempt) {
    HPM_TRY(t.cnt.ensure(sizeof(int) * level_grid, st));
    HPM_TRY(t.off.ensure(sizeof(int) * (cap + 1), st));
    HPM_TRY(t.bnd.ensure(sizeof(int) * 8 * cap, st));
    {
      const int64_t h0[2] = {0, nroot};
      HPM_CUDA(cudaMemcpyAsync(lvl, h0, sizeof(h0), cudaMemcpyHostToDevice, st));
      if (D + 2 > 2) HPM_CUDA(cudaMemsetAsync(lvl + 2, 0, sizeof(int64_t) * D, st));
      HPM_CUDA(cudaMemsetAsync(t.counters.as<int>() + 96, 0, sizeof(int) * 2, st));  // grid barrier
    }
    if (D > 0) {
      LevelArgs la;
      la.lvl = lvl;
      la.depth = D;
      la.leaf_max = pl->opts.leaf_max;
      la.cap = cap;
      la.flags = t.box_flags.as<uint8_t>();
      la.key = t.box_key.as<uint64_t>();
      la.beg = t.box_beg.as<int>();
      la.end = t.box_end.as<int>();
      la.parent = t.box_parent.as<int>();
      la.child = t.box_child.as<int>();
      la.nb = t.box_nb.as<int>();
      la.skeys = skeys;
      la.bnd = t.bnd.as<int>();
      la.off = t.off.as<int>();
      la.bsum = t.cnt.as<int>();
      la.counters = t.counters.as<int>();
      la.err = t.err.as<int>();
      la.gb = reinterpret_cast<GridBar *>(t.counters.as<int>() + 96);
      void *args[] = {&la};
      // One level kernel on a device at a time, whatever the stream: two
      // cooperative grids that each hold part of the GPU could wait on each
      // other's blocks. Each launch waits for the previous one on the same
      // device to finish (one event per device).
      static std::mutex mu;
      static cudaEvent_t last_ev[kMaxDevices] = {};
      int dev = 0;
      HPM_CUDA(cudaGetDevice(&dev));
      if (dev < 0 || dev >= kMaxDevices) return HPM_ERR_UNSUPPORTED;
      std::lock_guard<std::mutex> lock(mu);
      cudaEvent_t &last = last_ev[dev];
      if (!last) HPM_CUDA(cudaEventCreateWithFlags(&last, cudaEventDisableTiming));
      HPM_CUDA(cudaStreamWaitEvent(st, last, 0));
      HPM_CUDA(cudaLaunchCooperativeKernel((const void *)k_levels, dim3(level_grid), dim3(kThreads), args, 0, st));
      HPM_LAUNCHED(&launches);
      HPM_CUDA(cudaEventRecord(last, st));
    }
    // level offsets at 0 (at most 8 (kMaxDepth + 2) bytes), the error word
    // at 256, the per-level counts at 512 of the pinned buffer
    static_assert(8 * (kMaxDepth + 2) <= 256 && 512 + sizeof(int) * 64 <= kPinBytes, "read-back layout");
    int herr = 0;
    HPM_CUDA(cudaMemcpyAsync(hp, lvl, sizeof(int64_t) * (D + 2), cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaMemcpyAsync(hp + 256, t.err.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaMemcpyAsync(hp + 512, t.counters.p, sizeof(int) * 64, cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaStreamSynchronize(st));
    memcpy(pl->lvl_off.data(), hp, sizeof(int64_t) * (D + 2));
    memcpy(&herr, hp + 256, sizeof(int));
    memcpy(hc, hp + 512, sizeof(int) * 64);
    if (herr & kErrDomain) return HPM_ERR_OUT_OF_DOMAIN;
    if (herr & kErrTimeout) return HPM_ERR_TIMEOUT;
    if (!(herr & kErrCapacity)) break;
    if (attempt >= 8) return HPM_ERR_OOM;
    // more room, then the levels again (the roots are kept; per-level counts
    // and the error word are reset)
    cap *= 2;
    HPM_TRY(ensure_boxes(t, cap, st));
    HPM_TRY(ensure_scan_ctl(t.scan_buf, scan_tiles(cap + 1), t.err.as<int>(), st, &t.scan));
    HPM_CUDA(cudaMemsetAsync(t.err.p, 0, sizeof(int), st));
    HPM_CUDA(cudaMemsetAsync(t.counters.as<int>() + 1, 0, sizeof(int) * 31, st));
    HPM_CUDA(cudaMemsetAsync(t.counters.as<int>() + 33, 0, sizeof(int) * 31, st));
  }
  if (D == 0) pl->lvl_off[1] = nroot;  // the roots are the only boxes
  pl->nbox = pl->lvl_off[D + 1];
  {
    // what this build needed of the box arrays and the level scratch (their
    // capacity was estimated beforehand, or kept from a larger build)
    const size_t nb = (size_t)std::max<int64_t>(pl->nbox, 1);
    t.box_key.used = sizeof(uint64_t) * nb;
    t.box_beg.used = t.box_end.used = t.box_parent.used = sizeof(int) * nb;
    t.box_flags.used = (nb + 15) & ~size_t(15);
    t.box_child.used = sizeof(int) * 8 * nb;
    t.box_nb.used = sizeof(int) * 27 * nb;
    t.bnd.used = std::max<size_t>(sizeof(int) * 8 * nb, sizeof(int) * ((size_t)nprob + 1));
  }
  {
    // child maps of the deepest level are never filled: mark them empty
    const int64_t b = pl->lvl_off[D], e = pl->lvl_off[D + 1];
    if (e > b) HPM_CUDA(cudaMemsetAsync(t.box_child.as<int>() + b * 8, 0xff, sizeof(int) * 8 * (e - b), st));
  }

  // per-level counts of cells and leaves (read back above)
  int depth_reached = 0;
  int64_t ncell = 0, nleaf = 0;
  for (int l = 0; l <= D; ++l) {
    ncell += hc[l];
    nleaf += hc[32 + l];
    if (hc[l] > 0) depth_reached = l;
  }
  pl->depth_reached = depth_reached;
  pl->ncell = ncell;
  pl->tgt_lvl_off.assign(D + 2, 0);
  pl->leaf_lvl_off.assign(D + 2, 0);
  for (int l = 0; l <= D; ++l) {
    pl->tgt_lvl_off[l + 1] = pl->tgt_lvl_off[l] + (l >= 2 ? hc[l] : 0);
    pl->leaf_lvl_off[l + 1] = pl->leaf_lvl_off[l] + hc[32 + l];
  }

  // work lists: targets (cells at level >= 2), leaves, P2G boxes (level >= 2,
  // not expanded), parents of the targets (internal cells at levels >= 1); the
  // sizes of the first, second and fourth follow from the per-level counts of
  // cells and leaves, the P2G count is read back with the near-field counts
  const int64_t off2 = D >= 2 ? pl->lvl_off[2] : pl->nbox;
  {
    int64_t cells2 = 0, internal1 = 0;
    for (int l = 1; l <= D; ++l) {
      const int64_t internal = (int64_t)hc[l] - hc[32 + l];
      internal1 += internal;
      if (l >= 2) cells2 += hc[l];
    }
    pl->ntgt = cells2;
    pl->nleaf = nleaf;
    pl->np2g = -1;  // counted on the device (boxes at level >= 2 that are not expanded)
    pl->npar = internal1;
  }
  {
    // the four work lists (totals to counters[70..73]) in three launches
    const int64_t nb = pl->nbox > 0 ? pl->nbox : 1;
    const int nblk = (int)((pl->nbox + kThreads - 1) / kThreads);
    const int64_t off1 = D >= 1 ? pl->lvl_off[1] : pl->nbox;
    HPM_TRY(t.tgt_box.ensure(sizeof(int) * nb, st));
    HPM_TRY(t.leaf_box.ensure(sizeof(int) * nb, st));
    HPM_TRY(t.p2g_box.ensure(sizeof(int) * nb, st));
    HPM_TRY(t.par_box.ensure(sizeof(int) * nb, st));
    if (nblk > 0) {
      HPM_TRY(t.cnt.ensure(sizeof(int) * 4 * nblk, st));
      HPM_TRY(t.off.ensure(sizeof(int) * (4 * nblk + 1), st));
      k_lists_count<<<nblk, kThreads, 0, st>>>(pl->nbox, off2, off1, t.box_flags.as<uint8_t>(), nblk,
                                               t.cnt.as<int>());
      HPM_LAUNCHED(&launches);
      HPM_TRY(exclusive_scan_i32(t.cnt.as<int>(), t.off.as<int>(), 4 * (int64_t)nblk, t.off.as<int>() + 4 * nblk,
                                 t.scan, st, &launches));
      k_lists_write<<<nblk, kThreads, 0, st>>>(pl->nbox, off2, off1, t.box_flags.as<uint8_t>(), nblk,
                                               t.off.as<int>(), t.off.as<int>() + 4 * nblk, t.tgt_box.as<int>(),
                                               t.leaf_box.as<int>(), t.p2g_box.as<int>(), t.par_box.as<int>(),
                                               t.counters.as<int>() + 70);
      HPM_LAUNCHED(&launches);
    } else {
      HPM_CUDA(cudaMemsetAsync(t.counters.as<int>() + 70, 0, sizeof(int) * 4, st));
    }
  }
  // leaf of every particle
  HPM_TRY(t.pbox.ensure(sizeof(int) * (n > 0 ? n : 1), st));
  if (pl->nleaf) {
    k_particle_box<<<blocks_for(pl->nleaf), kThreads, 0, st>>>(pl->nleaf, t.leaf_box.as<int>(), t.box_beg.as<int>(),
                                                               t.box_end.as<int>(), t.pbox.as<int>());
    HPM_LAUNCHED(&launches);
  }
  // near-field work items
  {
    const int64_t nl = pl->nleaf;
    HPM_TRY(t.leaf_nitem.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.leaf_item0.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.leaf_part0.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.cnt.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.leaf_ns.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.big_leaf.ensure(sizeof(int) * (nl + 1), st));
    HPM_TRY(t.split_leaf.ensure(sizeof(int) * (nl + 1), st));
    // counters[76..77]: the near-zone pair count (64 bits), zeroed with the others
    k_leaf_work<<<blocks_for(nl), kThreads, 0, st>>>(nl, t.leaf_box.as<int>(), t.box_nb.as<int>(),
                                                     t.box_beg.as<int>(), t.box_end.as<int>(),
                                                     t.leaf_nitem.as<int>(), t.leaf_part0.as<int>(),
                                                     t.counters.as<int>() + 65, t.leaf_ns.as<int>(),
                                                     t.big_leaf.as<int>(), t.counters.as<int>() + 78,
                                                     t.split_leaf.as<int>(), t.counters.as<int>() + 79,
                                                     reinterpret_cast<unsigned long long *>(t.counters.as<int>() + 76));
    HPM_LAUNCHED(&launches);
    // items in leaf order (the near field takes them in index order: a leaf's
    // neighbours' particles are then still in cache for the next leaf)
    HPM_TRY(exclusive_scan_i32(t.leaf_nitem.as<int>(), t.leaf_item0.as<int>(), nl, t.counters.as<int>() + 80,
                               t.scan, st, &launches));
    int hv[17] = {0}, herr2[2] = {0, 0};
    HPM_CUDA(cudaMemcpyAsync(hp, t.counters.as<int>() + 64, sizeof(int) * 17, cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaMemcpyAsync(hp + 256, t.err.as<int>(), sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    HPM_CUDA(cudaStreamSynchronize(st));
    memcpy(hv, hp, sizeof(int) * 17);
    memcpy(herr2, hp + 256, sizeof(int) * 2);
    if (herr2[1] & kErrTimeout) {
      // a bounded wait of an earlier solve on this plan ran out: report it once
      HPM_CUDA(cudaMemsetAsync(t.err.as<int>() + 1, 0, sizeof(int), st));
      return HPM_ERR_TIMEOUT;
    }
    if (herr2[0] & kErrTimeout) return HPM_ERR_TIMEOUT;
    pl->nitem = hv[16];
    pl->npart = hv[1];
    pl->nbig = hv[14];
    pl->nsplit = hv[15];
    {
      unsigned long long pairs = 0;
      memcpy(&pairs, hv + 12, sizeof(pairs));
      pl->npairs = (int64_t)pairs;
    }
    pl->np2g = hv[8];
    // the work-list sizes the host derived must be what the device selected
    if (hv[6] != pl->ntgt || hv[7] != pl->nleaf || hv[9] != pl->npar) {
      fprintf(stderr, "hpm: work-list sizes disagree (device %d %d %d, host %lld %lld %lld)\n", hv[6], hv[7],
              hv[9], (long long)pl->ntgt, (long long)pl->nleaf, (long long)pl->npar);
      return HPM_ERR_INVALID_ARG;
    }
    HPM_TRY(t.item_leaf.ensure(sizeof(int) * (pl->nitem + 1), st));
    HPM_TRY(t.item_s0.ensure(sizeof(int) * (pl->nitem + 1), st));
    HPM_TRY(t.item_s1.ensure(sizeof(int) * (pl->nitem + 1), st));
    HPM_TRY(t.item_t.ensure(sizeof(int) * (pl->nitem + 1), st));
    k_fill_items<<<blocks_for(nl), kThreads, 0, st>>>(nl, t.leaf_box.as<int>(), t.leaf_ns.as<int>(),
                                                      t.box_beg.as<int>(), t.box_end.as<int>(),
                                                      t.leaf_nitem.as<int>(), t.leaf_item0.as<int>(),
                                                      t.item_leaf.as<int>(), t.item_s0.as<int>(),
                                                      t.item_s1.as<int>(), t.item_t.as<int>());
    HPM_LAUNCHED(&launches);
  }
  HPM_TRY(t.box_tgt.ensure(sizeof(int) * (pl->nbox > 0 ? pl->nbox : 1), st));
  HPM_CUDA(cudaMemsetAsync(t.box_tgt.p, 0xff, sizeof(int) * pl->nbox, st));
  if (pl->ntgt) {
    k_box_tgt<<<blocks_for(pl->ntgt), kThreads, 0, st>>>(pl->ntgt, t.tgt_box.as<int>(), t.box_tgt.as<int>());
    HPM_LAUNCHED(&launches);
  }
  if (pl->ntgt && !use_tc_m2l(pl)) {
    // per-target 6^3 blocks: read by the FFT-form source-to-target kernel only
    // (the tensor-core form builds its own per-parent tiles below)
    HPM_TRY(t.tgt_blk.ensure(sizeof(int) * 216 * pl->ntgt, st));
    HPM_TRY(t.tgt_info.ensure(sizeof(int) * pl->ntgt, st));
    LevelOffsets lo{};
    lo.nlev = D + 1;
    for (int l = 0; l <= D + 1; ++l) lo.off[l] = pl->lvl_off[l];
    k_target_blocks<<<blocks_for(27 * pl->ntgt), kThreads, 0, st>>>(
        pl->ntgt, t.tgt_box.as<int>(), t.box_parent.as<int>(), t.box_nb.as<int>(), t.box_child.as<int>(),
        t.box_key.as<uint64_t>(), off2, lo, t.tgt_blk.as<int>(), t.tgt_info.as<int>());
    HPM_LAUNCHED(&launches);
  }
  {
    // parents per level (internal cells = cells - leaves) for the tensor-core tiles
    std::vector<int64_t> par_per_level(D + 2, 0);
    for (int l = 1; l <= D; ++l) par_per_level[l] = hc[l] - hc[32 + l];
    HPM_TRY(tc_build_tiles(pl, par_per_level, st, &launches));
  }
  pl->stats.launches = launches;
  pl->built = true;
  return HPM_OK;
}

}  // namespace hpm
