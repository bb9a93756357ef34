// Internal declarations shared by the translation units of libhpm.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/hpm.h"

namespace hpm {

constexpr int kMaxNg = 8;
constexpr int kMaxDepth = 21;
constexpr int kMortonBits = 21;

// Box flags (a "box" is a nonempty dyadic box of some level that the solve
// needs: every real tree cell, plus the virtual boxes inside coarser leaves
// that lie in the parent neighbourhood of some internal cell).
enum : uint8_t {
  kReal = 1,      // a cell of the tree
  kInternal = 2,  // a cell that splits
  kLeaf = 4,      // a cell that does not split
  kExpand = 8,    // its children are needed (it neighbours an internal cell)
};

// Device error word bits.
enum : int { kErrDomain = 1, kErrCapacity = 2, kErrTimeout = 4 };

// Near-field table of a user kernel: 32 cubic segments per octave of r_u^2
// (r_u = distance / domain side) over [2^-64, 2^2); see green.cu.
constexpr int kNearTabE0 = -64;
constexpr int kNearTabOctaves = 66;
constexpr int kNearTabSeg = 32;

// Radix sort and single-pass scan sizing (sort.cu): elements per sort tile,
// digits per pass, elements per scan tile. The no-allocation sort sizes its
// static scratch from these.
constexpr int kSortTileElems = 4096;
constexpr int kRadixDigits = 256;
constexpr int kScanTileElems = 2048;
// ints of histogram and offsets radix_sort_pairs needs for n elements
constexpr int64_t sort_scratch_ints(int64_t n) {
  return 2 * (int64_t)kRadixDigits * ((n + kSortTileElems - 1) / kSortTileElems);
}
// scan tiles (status words) of a scan over n elements
constexpr int64_t scan_tiles_of(int64_t n) { return (n + kScanTileElems - 1) / kScanTileElems; }

// Near-field work item size: pairs per warp-sized item (and at least this many
// sources per item).
constexpr int64_t kP2PPairsPerItem = 16384;
constexpr int kP2PMinSources = 32;
// Leaves of more particles than this are split by targets instead (items of
// 32 targets against all the leaf's near sources, no partial sums)
constexpr int kP2PSplitTargets = 64;
// Leaves split over more items than this have their partial sums added by a
// block each (lanes over items) instead of a warp each (lanes over targets)
constexpr int kP2PCombineWarp = 32;

const char *set_cuda_error(cudaError_t e);

// Devices a process may use the library on (per-device caches below).
constexpr int kMaxDevices = 64;

// A value set up once per device (a function attribute, an occupancy, the
// SM count), under a lock: the serving loop's workers and callers on other
// devices share these.
struct DeviceCache {
  std::mutex mu;
  int value[kMaxDevices] = {};
  bool ready[kMaxDevices] = {};
};

// Device memory pool owned by the library on the current device (created on
// first use, kept until the process exits). Its release threshold keeps freed
// blocks for reuse between solves; the device's default pool, which other
// code in the caller's process may use, is left as it is.
hpm_status lib_pool(cudaMemPool_t *out);
// Stream-ordered allocation from that pool.
hpm_status lib_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Grow-only device buffer on the library's stream-ordered pool.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  size_t used = 0;  // the largest size asked for since the plan's last tree build began
  hpm_status ensure(size_t bytes, cudaStream_t s, bool keep = false);
  void release(cudaStream_t s);
  template <class T> T *as() const { return static_cast<T *>(p); }
};

// control words of the single-pass scan (a buffer of their own, zeroed when
// allocated): the tile ticket, one status word per tile, the error word
struct ScanCtl {
  unsigned *ticket = nullptr;
  unsigned long long *status = nullptr;
  int64_t tiles = 0;
  int *err = nullptr;
};

// Constant tables handed to kernels by value.
struct GridletTables {
  int ng;
  float node[kMaxNg];                // x_j = (j + 1/2)/Ng - 1/2
  float t1[2][kMaxNg][kMaxNg];       // T^{s}_{pq} = ell_p((a_s + x_q)/2), a_0 = -1/2, a_1 = +1/2
  float t1lo[2][kMaxNg][kMaxNg];     // T^{s}_{pq} - t1 (the rest of the FP64 value)
  double node_d[kMaxNg];
  double inv_den_d[kMaxNg];          // 1 / prod_{k != j} (x_j - x_k)
  double inv_den_u[kMaxNg];          // the same for the nodes 2 Ng x_j = 2j + 1 - Ng (integers)
  float inv_den[kMaxNg];
  float node_lo[kMaxNg];             // x_j - node[j], and 1 / prod(...) - inv_den[j]: the
  float inv_den_lo[kMaxNg];          // double-float rests of the FP64 values
};

struct TreeDev {
  // sorted particles
  DevBuf keys, keys_alt, perm, perm_alt;
  DevBuf spm;        // sorted particles: float4 unit-cube position hi (x, y, z, m) then lo (x, y, z, 0)
  // boxes, all levels, level-major, Morton order within a level
  DevBuf box_key, box_beg, box_end, box_parent, box_flags, box_child, box_nb;
  DevBuf cnt, off, bnd;   // per-box scratch for child counting
  // work lists
  DevBuf tgt_box, box_tgt, leaf_box, p2g_box, par_box;
  DevBuf pbox;       // leaf box of every sorted particle
  // interaction zone of every target as its 6^3 parent block: row of each box's
  // effective masses, -1 where empty, outside the domain or in the near zone;
  // and (level << 3 | child octant) per target
  DevBuf tgt_blk, tgt_info;
  // Ng = 4 tensor-core source-to-target: per tile of 256 parents of one level,
  // the rows of the 216 boxes of each parent's 6^3 block ([216][256], -1 where
  // empty) and the targets of its 8 children ([256][8], -1 where absent)
  DevBuf tc_rows, tc_tgt;
  // near-field work items: each leaf's concatenated near sources split into
  // items of bounded pair count
  // item_t: first target of a target-split item (32 targets), -1 for an item
  // that covers all the leaf's targets
  // big_leaf / split_leaf: leaves split over sources into more than
  // kP2PCombineWarp items / into 2 .. kP2PCombineWarp items (order not fixed)
  DevBuf item_leaf, item_s0, item_s1, item_t, leaf_nitem, leaf_item0, leaf_part0, leaf_ns, big_leaf, split_leaf;
  DevBuf err;        // int error word
  DevBuf lvl_dev;    // box offsets per level on the device (int64, max_depth + 2)
  DevBuf offsets;    // problem offsets of a batched build (int64, nprob + 1)
  DevBuf counters;   // small device counters
  DevBuf scan_buf;   // control words of the single-pass scan
  ScanCtl scan;
};

struct SolveDev {
  DevBuf grid;       // effective masses, row = box - lvl_off[2], Ng^3 floats
  DevBuf m2l_raw;    // source-to-target values per target, Ng^3
  DevBuf loc;        // local gridlets per target, Ng^3 deviations
  DevBuf locc;       // local constant per target
  DevBuf m2lc;       // constant part of each target's source-to-target values
  DevBuf far;        // far field per sorted particle: float4 (phi, ax, ay, az)
  DevBuf part;       // near-field partial sums of leaves split over several items
  DevBuf m2l_scratch;
  DevBuf work;       // near-field item counter (zeroed before each launch)
  // Ng = 4 tensor-core path: effective masses as FP16 (hi, lo) planes at a
  // per-row scale, row scale exponents and total masses, the scale exponent of
  // each tile column (parent) and the zone mass of each of its 8 children
  DevBuf grid_hl, box_em, col_exp, zone_mass;  // box_em: (scale exponent, total mass bits) per row
  DevBuf level_amax;  // per (problem, level): largest |effective mass| (float bits)
};

}  // namespace hpm

struct hpm_plan_s {
  hpm_domain dom;
  int max_depth;
  int ng;
  hpm_green green;
  hpm_plan_opts opts;
  int device;
  hpm::GridletTables tab;
  // the target (local) gridlet: the same as tab, or with HPM_FLAG_EXTENDED_GRIDLET
  // widened by one node on each side (ng_loc = ng + 2 nodes per axis)
  hpm::GridletTables tab_loc;
  int ng_loc = 0;
  // the kernel on the gridlet lattice, FP64, per level l: G_l[n] = g(h_l sqrt(n)),
  // n = 0 .. lattice_nmax(Ng) (G_l[0] = G_l[1]); glat_stride values per level
  hpm::DevBuf glat;
  int64_t glat_stride = 0;
  std::vector<double> glat_host;
  // user kernels: near-field table, per segment 4 cubic coefficients of g then
  // 4 of F = -g'(r) / r_u (FP32)
  hpm::DevBuf near_tab;
  // Green transforms, reduced (P/2+1)^3 FP32 tables per level, scaled -1/P^3
  hpm::DevBuf ghat;
  int64_t ghat_level_stride;  // floats per level
  // mean of the periodic Green function per level, removed from the DC bin of
  // the stored transform and added back to each target's constant
  hpm::DevBuf gmean;
  // Green function transformed along x only, per level: K[kx][|dy|][|dz|] =
  // -(1/P) sum_dx (G - mean) cos(2 pi kx dx / P), kx in [0, P/2], |dy|,|dz| < 4 Ng
  hpm::DevBuf kx_green;
  int64_t kx_green_stride = 0;      // floats per level
  // Ng = 4: the Green transform inverse-transformed along z only, per level:
  // K2[kx][|ky|][|dz|] = sum_kz G^(kx, ky, kz) cos(2 pi kz dz / P) (scaled -1/P^3,
  // DC removed), kx, |ky| in [0, P/2], |dz| < 4 Ng
  hpm::DevBuf kz_green;
  int64_t kz_green_stride = 0;
  // Ng = 4 tensor-core source-to-target: the dense matrices W_l of levels
  // 2..max_depth as TF32 (hi, lo) tiles in streaming order, and the tiles of
  // the built tree (first tile of each target level)
  hpm::DevBuf tc_w;
  hpm::DevBuf tc_wexp;                // per level and row: power-of-two scale exponent
  hpm::DevBuf tc_mean;                // per target level and child: mean of row (o, 0)
  std::vector<double> tc_mean_host;
  int64_t tc_ntiles = 0;
  int tc_tile_n = 256;  // parents per tile of the last tree build
  std::vector<int64_t> tc_tile_off;
  // tree
  hpm::TreeDev t;
  hpm::SolveDev s;
  bool built = false;
  int64_t n = 0;
  int nprob = 1;                   // problems in the built tree (batched builds)
  std::vector<int64_t> prob_off;   // host copy of the problem offsets
  std::vector<int64_t> lvl_off;    // box offsets per level, size depth+2
  int depth_reached = -1;
  int64_t nbox = 0, ntgt = 0, nleaf = 0, np2g = 0, ncell = 0;
  int64_t nitem = 0, npart = 0;   // near-field work items, partial-sum rows
  int64_t npairs = 0;              // near-zone pairs (i, j), j != i
  int64_t nbig = 0;                // leaves split over more than kP2PCombineWarp items
  int64_t nsplit = 0;              // leaves split over 2 .. kP2PCombineWarp items
  int64_t npar = 0;                // internal cells at levels >= 1 (parents of targets)
  std::vector<int64_t> tgt_lvl_off;  // target offsets per level (levels 2..D)
  std::vector<int64_t> leaf_lvl_off;
  hpm_stats stats{};
  hpm_tuning tuning{};             // launch shapes (0 = default), see hpm_set_tuning
  int test_stall = 0;              // failure test hook (hpm_test_stall)
  long long test_wait_limit = 0;   // cycles per bounded wait in that test (0 = default)
  cudaEvent_t ev[12] = {};  // stage boundaries 0..7, tree 8..9, dense product kernel 10..11
  // pinned host memory for the tree build's small read-backs (copies into
  // pageable memory would each wait for their own round trip)
  unsigned char *h_pin = nullptr;
  bool events_ready = false;
  hpm::DevBuf host_io_pos, host_io_mass, host_io_phi, host_io_acc;
  // hpm_solve_host: the masses' host-to-device copy runs on a stream of its
  // own, after the positions' copy, while the tree is built
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_ev[2] = {};
  hpm::DevBuf batch_desc;          // device copy of a batch's problem table and offsets
};

namespace hpm {
// tree.cu
hpm_status launch_morton_keys(const hpm_domain &dom, int depth, const double *d_pos, int64_t n,
                              uint64_t *d_keys, int *d_err, cudaStream_t st);
hpm_status build_tree(hpm_plan_s *pl, const double *d_pos, int64_t n, const int64_t *h_offsets, int nprob,
                      cudaStream_t st);
// sort.cu
int64_t scan_tiles(int64_t n);
hpm_status ensure_scan_ctl(DevBuf &buf, int64_t tiles, int *err, cudaStream_t st, ScanCtl *out);
// (wide_digits: 9-bit digits where they take fewer passes; the scratch then
// needs 512 counters per tile of kSortTileElems, not kRadixDigits)
hpm_status radix_sort_pairs(uint64_t *&keys, uint64_t *&keys_alt, uint32_t *&vals,
                            uint32_t *&vals_alt, int64_t n, int bits, DevBuf &scratch, const ScanCtl &ctl,
                            cudaStream_t st, int64_t *launches, bool wide_digits = false);
hpm_status exclusive_scan_i32(const int *in, int *out, int64_t n, int *d_total, const ScanCtl &ctl,
                              cudaStream_t st, int64_t *launches);
// green.cu
double green_g(const hpm_green &g, double r);
int64_t lattice_nmax(int ng);
hpm_status build_lattice(hpm_plan_s *pl, cudaStream_t st);
hpm_status build_near_table(hpm_plan_s *pl, cudaStream_t st);
// solve.cu
// warps (gridlets) per CTA of the Ng = 4 child-to-parent and parent-to-child kernels
inline int gridlet_warps(const hpm_plan_s *pl) {
  const int w = pl->tuning.gridlet_warps;
  return (w == 2 || w == 4) ? w : 8;
}
hpm_status solve(hpm_plan_s *pl, const double *d_pos, const double *d_mass, float *d_phi,
                 float *d_acc, cudaStream_t st);
hpm_status precompute_green(hpm_plan_s *pl, cudaStream_t st);
hpm_status batch_gather(const hpm_problem *d_desc, const int64_t *d_off, int nprob, int64_t n, double *pos,
                        double *mass, cudaStream_t st);
hpm_status batch_scatter(const hpm_problem *d_desc, const int64_t *d_off, int nprob, int64_t n, const float *phi,
                         const float *acc, cudaStream_t st);
// m2l.cu
hpm_status launch_m2l(hpm_plan_s *pl, cudaStream_t st, int64_t *launches);
// m2l_tc.cu
int sm_count();
bool use_tc_m2l(const hpm_plan_s *pl);
hpm_status tc_precompute(hpm_plan_s *pl, cudaStream_t st);
hpm_status tc_build_tiles(hpm_plan_s *pl, const std::vector<int64_t> &par_per_level, cudaStream_t st,
                          int64_t *launches);
hpm_status launch_m2l_tc(hpm_plan_s *pl, cudaStream_t st, int64_t *launches);
// block order of the dense source-to-target kernel: 1 tile-major, 2 row-block-major
int m2l_block_order(const hpm_plan_s *pl);
void plan_bytes(hpm_plan_s *pl, int64_t *tables, int64_t *work);
void reset_work_need(hpm_plan_s *pl);
int m2l_tile_parents(const hpm_plan_s *pl);
}  // namespace hpm

#define HPM_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      hpm::set_cuda_error(e_);                          \
      return e_ == cudaErrorMemoryAllocation ? HPM_ERR_OOM : HPM_ERR_CUDA; \
    }                                                   \
  } while (0)

#define HPM_TRY(call)                 \
  do {                                \
    hpm_status s_ = (call);           \
    if (s_ != HPM_OK) return s_;      \
  } while (0)

namespace hpm {
// The cached value of `c` for the current device, computed by `compute(int *)`
// (an hpm_status-returning callable) the first time.
template <class F>
hpm_status device_cached(DeviceCache &c, F &&compute, int *out) {
  int dev = 0;
  HPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return HPM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(c.mu);
  if (!c.ready[dev]) {
    int v = 0;
    HPM_TRY(compute(&v));
    c.value[dev] = v;
    c.ready[dev] = true;
  }
  *out = c.value[dev];
  return HPM_OK;
}
}  // namespace hpm

#define HPM_LAUNCHED(counter)                           \
  do {                                                  \
    cudaError_t e_ = cudaGetLastError();                \
    if (e_ != cudaSuccess) {                            \
      hpm::set_cuda_error(e_);                          \
      return HPM_ERR_CUDA;                              \
    }                                                   \
    if (counter) ++*(counter);                          \
  } while (0)
