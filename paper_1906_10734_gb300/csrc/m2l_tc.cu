// Source-to-target values for Ng = 4 as a dense product on the tensor cores.
//
// The interaction zones of the 8 children of one parent all lie in the 6^3
// block of the parent's neighbours' children (Sec. 1), and on the level-l grid
// the convolution of Sec. 2.1 is translation invariant, so the values at the
// children's 8 x 64 nodes are one fixed matrix W_l (512 x 216*64 per level)
// times the 216 gridlets of that block:
//
//   Phi[(o, i)][P] = sum_{s, j} W_l[(o, i)][(s, j)] rho_{block(P, s)}[j],
//   W_l[(o, i)][(s, j)] = -g(h_l |y_{o,i} - y_{s,j}|), zero where slot s is in
//   the near zone of child o.
//
// This is the same convolution the FFT path evaluates (exactly, up to
// rounding), written as a GEMM with the parents as the N dimension. Precision:
// each row of W and each parent's column of rho is scaled by a power of two
// (exact) so that its largest entry lies in [2^13, 2^14), then split into FP16
// pairs (x = hi + lo, 22 significant bits; entries far below the row's or
// column's largest keep an absolute error under 2^-24 of the scaled unit), and
// three products hi*hi + hi*lo + lo*hi are accumulated in FP32 in tensor
// memory; the scales are removed when the values are written. The column
// scale is shared by all boxes of one level of one problem: a box whose
// largest |mass| is 2^-k of the level's largest keeps 22 bits for k <= 17 and
// loses bits gradually beyond (its contribution shrinks in proportion). The tensor
// core's accumulation drops low bits, so the accumulator is drained every
// kBlockChunks K-chunks into a round-to-nearest FP32 total held in the drain
// warps' registers, which keeps the chain short; two accumulator buffers
// alternate, so the MMAs of one block run while the previous block drains.
// Rows (o, i >= 1) hold deviations from node 0 of the child, the (constant,
// deviations) split of the local expansion that the FFT path also produces;
// row (o, 0) holds its entries minus their mean m_o over the interaction zone,
// and m_o times the zone's total mass (summed separately in compensated FP32)
// is added back to the constant, which keeps that row's sum free of a large
// same-sign running total.
//
// A pair of CTAs (a cluster of 2 on neighbouring SMs) computes 256 rows (4
// children) for 256 parents of one level with tcgen05.mma.cta_group::2: each
// CTA holds 128 rows of W and 128 of the parents in shared memory and 128 rows
// of the result in its tensor memory, so each SM loads half of the gathered
// parents the pair's MMAs read. Per CTA:
//   warp 0       bulk-copies the W tiles of each slot (pre-swizzled in HBM)
//   warp 1       allocates tensor memory (both CTAs) and, in the leader,
//                issues the MMAs and their commits to both CTAs' barriers
//   warps 2, 3   in the peer, tell the leader when each stage has landed
//   warps 4-7    gather this CTA's 128 parents' source gridlets with
//                cp.async, one z plane each (FP16 pairs split once per solve
//                by k_split, at one power-of-two scale per problem and
//                level, so a parent's column needs no rescaling)
//   warps 8-15   drain this CTA's accumulator rows and write the targets'
//                values
// Every wait is bounded; a wait that runs out sets kErrTimeout in the error
// word and the CTA leaves its loops.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "hpm_internal.cuh"

namespace hpm {
namespace tc {

constexpr int kSlots = 216;                     // 6^3 source block
constexpr int kKC = 16;                         // K elements per chunk (a 64-byte row of FP16 hi, lo)
constexpr int kRows = 128;                      // rows of W per CTA
constexpr int kRowBytes = 2 * kKC * 2;          // one tile row: 16 hi then 16 lo FP16 values
constexpr int kABytes = kRows * kRowBytes;      // W tile of one K-chunk: 8 KB
constexpr int kScaleTop = 14;                   // scaled maxima lie in [2^13, 2^14)
constexpr int kNoExp = 1 << 20;                 // exponent of a row without mass


// Sizes per gridlet order. K runs over the 216 source slots, each slot's
// gridlet padded to a multiple of 16 nodes (kCPS K-chunks per slot); the rows
// of W are the 8 children's nodes (kRowsReal), padded to 128-row blocks, one
// per CTA (pairs of CTAs take consecutive blocks of one tile). Ng = 4: 4
// chunks per slot, 864 per tile, 512 rows in 4 blocks; Ng = 6: 216 nodes in
// 14 chunks, 3024 per tile, 1728 rows in 14 blocks (64 padding rows).
template <int NG, int TN = (NG == 4 ? 256 : 128)>
struct Cfg {
  // The tensor core's accumulation truncates: each MMA's sum is added to the
  // accumulator rounded toward zero, and the error grows with the number of
  // additions since the last drain into the round-to-nearest FP32 totals in
  // registers. The K sum of the deviation rows cancels heavily, and more so
  // at higher order, so the accumulator is drained more often there (every 16
  // K-chunks at Ng = 4, every 8 at Ng = 6).
  static constexpr int kBlockChunks = NG == 4 ? 16 : 8;
  // Parents per tile (the MMA's N) and the drain's running totals: at Ng = 4
  // 256 parents and FP32 totals (128 columns per drain thread in registers);
  // at Ng = 6 the K sum of the deviation rows is longer and cancels more, and
  // the FP32 additions of the drained blocks would dominate the error, so the
  // totals are compensated (two-sum errors gathered in bf16 terms), which
  // fits in registers for 64 columns per drain thread: 128 parents per tile.
  // At Ng = 4 the width is a launch shape (256, 224 or 192 parents): a
  // narrower tile spreads a level's parents over more CTA pairs, which fills
  // the last wave better when the tile count is just above a multiple of the
  // pairs that fit; each column's K sum is the same whatever the width.
  static constexpr int kTileN = TN;
  static constexpr bool kDfTotals = NG != 4;
  // K-chunks per pipeline stage: the stage's synchronisation (barrier waits
  // and commits of the issuing thread, a few hundred cycles) must stay below
  // the MMAs' time, 3 x 4 x 128 cycles at 256 parents; 128 parents need 8
  // chunks per stage for the same MMA time. Each CTA of a pair loads its own
  // 128 rows of W and half of the parents per stage.
  static constexpr int kStageChunks = NG == 4 ? 4 : 8;
  static constexpr int kStageABytes = kStageChunks * kABytes;   // W of a stage, one bulk copy
  static constexpr int kHalfN = kTileN / 2;                     // parents gathered by each CTA of a pair
  static constexpr int kCols = kTileN / 2;                      // columns per drain thread (2 warps per lane quadrant)
  static constexpr int kColGroup = kCols % 32 == 0 ? 32 : (kCols % 16 == 0 ? 16 : 8);  // columns per tensor-memory load of the FP32 drain
  // accumulator buffer x at tensor-memory column kAccStride x (the second
  // buffer starts at column 256 for every width, as at 256 parents)
  static constexpr int kAccStride = NG == 4 ? 256 : kTileN;
  static constexpr int kBBytes = kHalfN * kRowBytes;            // gathered tile of one K-chunk
  static constexpr int kStageBytes = kStageChunks * (kABytes + kBBytes);  // 4 W tiles, then 4 B tiles
  static constexpr int kStages = NG == 4 ? 3 : 2;               // 3 x 64 KB or 2 x 96 KB
  // 1 KB for aligning the stages, 8 KB of slack past the last one
  static constexpr int kSmem = kStages * kStageBytes + 1024 + 8192;
  // instruction descriptor, kind::f16: FP32 accumulator, FP16 A and B (format
  // 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24. The MMA spans a CTA
  // pair: M = 256 rows (128 in each CTA's shared and tensor memory), N = the
  // tile's parents (each CTA's B rows are half of them).
  static constexpr uint32_t kIdesc =
      (1u << 4) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)((2 * kRows) >> 4) << 24);
  static_assert(kTileN % 16 == 0 && kTileN <= 256 && kAccStride + kTileN <= 512, "MMA N and two accumulator buffers");
  static_assert(kCols % kColGroup == 0 && kHalfN % 8 == 0, "drain column groups, gather groups");
  static_assert(kBBytes % 512 == 0, "B tiles start on a 512-byte swizzle atom");
  static_assert(NG == 4 || TN == 128, "the compensated drain holds 64 columns per thread");
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static constexpr int kM3 = NG * NG * NG;                      // nodes per gridlet
  static constexpr int kCPS = (kM3 + kKC - 1) / kKC;            // K-chunks per source slot
  static constexpr int kChunks = kSlots * kCPS;                 // K-chunks per tile
  static constexpr int kRowsReal = 8 * kM3;                     // rows of W that exist
  static constexpr int kQuarters = (kRowsReal + kRows - 1) / kRows;   // 128-row blocks (CTAs per tile)
  static constexpr int kSlotUses = kChunks / kStageChunks;      // stage uses per CTA
  static constexpr int kBlocks = kChunks / kBlockChunks;        // accumulator drains per CTA
  static constexpr int64_t kLevelBytes = (int64_t)kQuarters * kChunks * kABytes;  // W bytes per level
  static_assert(kChunks % kBlockChunks == 0, "drain blocks tile the K loop");
  static_assert(kBlockChunks % kStageChunks == 0, "drain blocks hold whole stages");
  static_assert(kQuarters % 2 == 0, "CTA pairs");
  static_assert(kCPS >= 4, "a gather warp's next chunk (4 chunks on) is in the same or the next slot");
};

// 4 warpgroups: 0 = W copy (warp 0), tensor memory and MMA issue (warp 1),
// relays of the peer's stages (warps 2, 3); 1 = gather; 2, 3 = drain. The drain warps keep the running totals in
// registers (128 per thread), so they take registers from the other two:
// 128 x (kRegsCtl + kRegsGather) + 2 x 128 x kRegsHigh = 512 x 128 = the
// launch's total.
constexpr int kWarps = 16, kThreads = kWarps * 32;
constexpr int kProdWarp0 = 4, kEpiWarp0 = 8;
constexpr int kGatherWarps = kEpiWarp0 - kProdWarp0;  // chunk g, g + 4, ... of every stage
constexpr int kLaunchRegs = 128, kRegsCtl = 40, kRegsGather = 104, kRegsHigh = 184;
static_assert(128 * kRegsCtl + 128 * kRegsGather + 2 * 128 * kRegsHigh == kThreads * kLaunchRegs, "register split");
static_assert(kGatherWarps == 4, "gather warp g copies K-chunks g, g + 4, ... of every stage");
// setmaxnreg: .dec only lowers, .inc only raises; counts are multiples of 8 in [24, 256]
static_assert(kRegsCtl <= kLaunchRegs && kRegsGather <= kLaunchRegs && kRegsHigh >= kLaunchRegs, "dec / inc");
static_assert(kRegsCtl % 8 == 0 && kRegsGather % 8 == 0 && kRegsHigh % 8 == 0 && kRegsCtl >= 24 && kRegsHigh <= 256,
              "register counts");

struct Params {
  const unsigned char *w;  // W tables, level l at w + (l - 2) * Cfg<NG>::kLevelBytes
  const int *w_exp;        // per level (from 2) and row: the row's scale exponent
  const int *col_exp;      // per tile and parent: the column's scale exponent
  const unsigned char *hl; // per row and z plane: 16 hi then 16 lo FP16 values at its level's scale
  const float *zone_mass;  // per tile, parent and child: total mass of the child's zone
  const int *rows;         // per tile: [216][256] source row or -1
  const int *tgt;          // per tile: [256][8] target index or -1
  int64_t tile_off[kMaxDepth + 2];  // tiles of target level l start at tile_off[l]
  int64_t ntiles;
  int qmajor;              // block order: 0 tile-major (the row blocks of a tile are
                           // consecutive), 1 row-block-major (a pair of row blocks
                           // runs over every tile before the next pair)
  int nlev;                // target levels 0..nlev-1 (tiles only at l >= 2)
  float *out;              // per target Ng^3: deviations from node 0 (node 0 holds 0)
  float *outc;             // per target: the value at node 0
  int *err;
  long long wait_limit;    // cycles a barrier wait may take before it gives up
  int stall;               // test hook: the leader's MMA thread first waits on a barrier nothing arrives at
  double mean[kMaxDepth + 1][8];  // m_o per target level: mean of row (o, 0) over the zone
};
// (NG in the comments above: the gridlet order of the launch)

// ---------------------------------------------------------------------------
// PTX wrappers
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(su32(b)),
               "r"(bytes)
               : "memory");
}
// Bounded wait for the phase of the given parity: at most `limit` cycles
// (about 2^32 by default).
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  uint32_t done = 0;
  for (;;) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(b))
               : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16-byte global -> shared copy; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp16(uint32_t dst, const void *src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand with 64-byte swizzle: rows
// of 64 bytes, 8-row groups 512 bytes apart, descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the barrier at this offset in both CTAs of the pair once the MMAs
// issued so far have completed
__device__ __forceinline__ void mma_commit(uint64_t *b) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          su32(b)),
      "h"((unsigned short)3)
      : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive on the barrier at the same offset in CTA `cta` of the cluster,
// releasing this thread's earlier writes (and what it acquired) to it
__device__ __forceinline__ void bar_arrive_remote(uint64_t *b, uint32_t cta) {
  uint32_t ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(su32(b)), "r"(cta));
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(ra) : "memory");
}
// bounded wait that also acquires what the other CTA of the pair released
__device__ __forceinline__ bool bar_wait_cl(uint64_t *b, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  uint32_t done = 0;
  for (;;) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\tselp.u32 "
        "%0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

#define HPM_R32(a) \
  "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]), "=r"(a[8]), \
      "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15]), "=r"(a[16]),   \
      "=r"(a[17]), "=r"(a[18]), "=r"(a[19]), "=r"(a[20]), "=r"(a[21]), "=r"(a[22]), "=r"(a[23]), "=r"(a[24]),  \
      "=r"(a[25]), "=r"(a[26]), "=r"(a[27]), "=r"(a[28]), "=r"(a[29]), "=r"(a[30]), "=r"(a[31])
#define HPM_W32(a) \
  "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), "r"(a[8]), "r"(a[9]), \
      "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]), "r"(a[16]), "r"(a[17]),           \
      "r"(a[18]), "r"(a[19]), "r"(a[20]), "r"(a[21]), "r"(a[22]), "r"(a[23]), "r"(a[24]), "r"(a[25]),           \
      "r"(a[26]), "r"(a[27]), "r"(a[28]), "r"(a[29]), "r"(a[30]), "r"(a[31])

// 32 lanes x 32 consecutive columns of tensor memory (lane = thread of the warp)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : HPM_R32(v)
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      HPM_W32(v)
      : "memory");
}
// 32 lanes x 16 consecutive columns
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
// 32 lanes x 8 consecutive columns
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// exact power of two for |e| < 127
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// exponent that brings a largest magnitude m > 0 into [2^13, 2^14)
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return min(max(kScaleTop - e, -120), 120);
}
__device__ __forceinline__ uint32_t pack_h2(__half a, __half b) {
  return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

// Byte offset of 16-byte chunk k (0..3) of row r in a K-major tile of 64-byte
// rows with 64-byte swizzle (chunk index XOR bits 1-2 of the row).
__host__ __device__ __forceinline__ int sw64(int r, int k) { return (r >> 3) * 512 + (r & 7) * 64 + ((k ^ ((r >> 1) & 3)) << 4); }

// ---------------------------------------------------------------------------
// Entry (row r of row block q, K-chunk c, node jj of the chunk) of W_l:
// -g(h |d|) for the child's node, minus the same for node 0 (rows of nodes
// >= 1) or minus the row mean m_o (node 0); zero in the near zone and in the
// padding (rows beyond the 8 children, nodes beyond a gridlet's Ng^3).
template <int NG>
__device__ __forceinline__ double w_entry(int q, int r, int c, int jj, const double *__restrict__ gl,
                                          const double *__restrict__ mean) {
  using C = Cfg<NG>;
  const int R = q * kRows + r;
  if (R >= C::kRowsReal) return 0.0;
  const int o = R / C::kM3, node = R - o * C::kM3;
  const int px = 2 + (o & 1), py = 2 + ((o >> 1) & 1), pz = 2 + (o >> 2);  // child in the 6^3 block
  const int s = c / C::kCPS, jn = kKC * (c - s * C::kCPS) + jj;           // source slot, node in its gridlet
  if (jn >= C::kM3) return 0.0;
  const int sx = s % 6, sy = (s / 6) % 6, sz = s / 36;
  if (max(abs(sx - px), max(abs(sy - py), abs(sz - pz))) <= 1) return 0.0;
  const int bx = NG * sx + jn % NG, by = NG * sy + (jn / NG) % NG, bz = NG * sz + jn / (NG * NG);  // grid units
  const int nx = node % NG, ny = (node / NG) % NG, nz = node / (NG * NG);
  const int dx = NG * px + nx - bx, dy = NG * py + ny - by, dz = NG * pz + nz - bz;
  double w = -gl[dx * dx + dy * dy + dz * dz];  // -g(h |d|), the level's lattice table
  if (node != 0) {
    const int ex = NG * px - bx, ey = NG * py - by, ez = NG * pz - bz;
    w += gl[ex * ex + ey * ey + ez * ez];
  } else {
    w -= mean[o];
  }
  return w;
}

// Largest |entry| of each row (as float bits, nonnegative floats order like
// their bits). One thread per (q, c, row).
template <int NG>
__global__ void k_w_rowmax(const double *__restrict__ gl, const double *__restrict__ mean, int *__restrict__ rowmax) {
  using C = Cfg<NG>;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)C::kQuarters * C::kChunks * kRows) return;
  const int r = (int)(i % kRows), c = (int)((i / kRows) % C::kChunks), q = (int)(i / ((int64_t)kRows * C::kChunks));
  double m = 0.0;
  for (int jj = 0; jj < kKC; ++jj) m = fmax(m, fabs(w_entry<NG>(q, r, c, jj, gl, mean)));
  if (m > 0.0) atomicMax(rowmax + q * kRows + r, __float_as_int((float)m));
}

// W_l in the order the kernel streams it: for each row block q and K-chunk c
// an 8 KB tile of 128 rows x (16 hi, 16 lo) FP16 values of the row-scaled
// entries, swizzled as the MMA reads it. One thread per (q, c, row); the c = 0
// threads also store the row exponents.
template <int NG>
__global__ void k_w_table(const double *__restrict__ gl, const double *__restrict__ mean, const int *__restrict__ rowmax,
                          unsigned char *__restrict__ out, int *__restrict__ w_exp) {
  using C = Cfg<NG>;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)C::kQuarters * C::kChunks * kRows) return;
  const int r = (int)(i % kRows), c = (int)((i / kRows) % C::kChunks), q = (int)(i / ((int64_t)kRows * C::kChunks));
  const int e = scale_exp(__int_as_float(rowmax[q * kRows + r]));
  if (c == 0) w_exp[q * kRows + r] = e;
  const double sc = ldexp(1.0, e);
  uint32_t hw[8], lw[8];
  for (int jj = 0; jj < kKC; jj += 2) {
    const double a = w_entry<NG>(q, r, c, jj, gl, mean) * sc, b = w_entry<NG>(q, r, c, jj + 1, gl, mean) * sc;
    const __half ah = __double2half(a), bh = __double2half(b);
    hw[jj / 2] = pack_h2(ah, bh);
    lw[jj / 2] = pack_h2(__double2half(a - (double)__half2float(ah)), __double2half(b - (double)__half2float(bh)));
  }
  unsigned char *tile = out + ((int64_t)q * C::kChunks + c) * kABytes;
  *reinterpret_cast<uint4 *>(tile + sw64(r, 0)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  *reinterpret_cast<uint4 *>(tile + sw64(r, 1)) = make_uint4(hw[4], hw[5], hw[6], hw[7]);
  *reinterpret_cast<uint4 *>(tile + sw64(r, 2)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  *reinterpret_cast<uint4 *>(tile + sw64(r, 3)) = make_uint4(lw[4], lw[5], lw[6], lw[7]);
}

// Source rows and target indices of every tile: tiles group the parents of one
// level (par_box is level-major), kTileN per tile, the last one padded with -1.
struct TileLevels {
  int64_t tile_off[kMaxDepth + 2];  // by target level
  int64_t par_off[kMaxDepth + 2];   // parents of target level l: par_box[par_off[l] .. par_off[l + 1])
  int nlev;
};

__global__ void k_tiles(int64_t ntiles, int kTileN, TileLevels tl, const int *__restrict__ par_box,
                        const int *__restrict__ nb, const int *__restrict__ child, const int *__restrict__ box_tgt,
                        int64_t off2, int *__restrict__ rows, int *__restrict__ tgt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ntiles * kTileN) return;
  const int64_t tile = i / kTileN;
  const int n = (int)(i % kTileN);
  int l = 2;
  while (l + 1 < tl.nlev && tl.tile_off[l + 1] <= tile) ++l;
  const int64_t pi = tl.par_off[l] + (tile - tl.tile_off[l]) * kTileN + n;
  int *rr = rows + tile * kSlots * kTileN + n;
  int *tt = tgt + (tile * kTileN + n) * 8;
  if (pi >= tl.par_off[l + 1]) {
    for (int s = 0; s < kSlots; ++s) rr[(int64_t)s * kTileN] = -1;
    for (int o = 0; o < 8; ++o) tt[o] = -1;
    return;
  }
  const int p = par_box[pi];
  // the 27 neighbours at once, then each one's 8 children as two 16-byte
  // loads (a box's child row is 32 contiguous bytes), all independent
  int q[27];
#pragma unroll
  for (int k = 0; k < 27; ++k) q[k] = __ldg(nb + (int64_t)p * 27 + k);
  const int4 *child4 = reinterpret_cast<const int4 *>(child);
#pragma unroll
  for (int k = 0; k < 27; ++k) {
    const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
    int4 c0 = make_int4(-1, -1, -1, -1), c1 = c0;
    if (q[k] >= 0) {
      c0 = __ldg(child4 + (int64_t)q[k] * 2);
      c1 = __ldg(child4 + (int64_t)q[k] * 2 + 1);
    }
    const int ch[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int bx = 2 * dx + (c & 1), by = 2 * dy + ((c >> 1) & 1), bz = 2 * dz + (c >> 2);
      rr[(int64_t)(bx + 6 * by + 36 * bz) * kTileN] = ch[c] >= 0 ? (int)(ch[c] - off2) : -1;
    }
  }
  for (int o = 0; o < 8; ++o) {
    const int ch = child[(int64_t)p * 8 + o];
    tt[o] = ch >= 0 ? box_tgt[ch] : -1;
  }
}

// Rows of the source grid belong to a level and a problem; the scale of a
// row is that of its (problem, level): the largest |effective mass| over the
// level's rows of that problem, brought into [2^13, 2^14).
struct RowLevels {
  int64_t off[kMaxDepth + 2];  // box offsets per level
  int nlev;
  int64_t off2;                // first box of level 2 (row 0)
};

__device__ __forceinline__ int row_scale_slot(const RowLevels &rl, const uint64_t *__restrict__ box_key, int64_t row) {
  const int64_t box = row + rl.off2;
  int l = 2;
  while (l + 1 < rl.nlev && rl.off[l + 1] <= box) ++l;
  const uint64_t p = box_key[box] >> (3 * l);  // problem index of a batched build (0 otherwise)
  return (int)p * rl.nlev + l;
}

// Effective masses of every row as FP16 pairs at the row's (problem, level)
// scale, in the order the gather copies them: per K-chunk (16 nodes) 16 hi
// then 16 lo values (64 bytes), nodes beyond Ng^3 zero; also the row's scale
// exponent (kNoExp without mass) and total mass. kL lanes per row (a power of
// two >= the chunks per row), one K-chunk each.
template <int NG>
__global__ void k_split(int64_t nrow, const float *__restrict__ grid, const uint64_t *__restrict__ box_key,
                        RowLevels rl, const int *__restrict__ amax, unsigned char *__restrict__ hl,
                        int2 *__restrict__ box_em) {
  using C = Cfg<NG>;
  constexpr int kL = C::kCPS <= 4 ? 4 : (C::kCPS <= 8 ? 8 : (C::kCPS <= 16 ? 16 : 32));
  static_assert(C::kCPS <= kL && C::kM3 % 4 == 0, "lanes per row");
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t row = i / kL;
  const int zq = (int)(i % kL);
  const bool live = row < nrow && zq < C::kCPS;
  float v[kKC];
  float m = 0.f, sum = 0.f;
#pragma unroll
  for (int k = 0; k < kKC; ++k) v[k] = 0.f;
  if (live) {
    const float4 *g = reinterpret_cast<const float4 *>(grid + row * C::kM3 + zq * kKC);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (zq * kKC + 4 * k < C::kM3) {
        const float4 a = g[k];
        v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = a.z; v[4 * k + 3] = a.w;
      }
    }
#pragma unroll
    for (int k = 0; k < kKC; ++k) {
      m = fmaxf(m, fabsf(v[k]));
      sum += v[k];
    }
  }
  // the row's chunks are kL consecutive lanes
#pragma unroll
  for (int o = 1; o < kL; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
#pragma unroll
  for (int o = 1; o < kL; o <<= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (!live) return;
  const int e = scale_exp(__int_as_float(amax[row_scale_slot(rl, box_key, row)]));
  const float sc = pow2f(e);
  uint32_t hw[8], lw[8];
#pragma unroll
  for (int k = 0; k < kKC; k += 2) {
    const float a = v[k] * sc, b = v[k + 1] * sc;
    const __half ah = __float2half_rn(a), bh = __float2half_rn(b);
    hw[k / 2] = pack_h2(ah, bh);
    lw[k / 2] = pack_h2(__float2half_rn(a - __half2float(ah)), __float2half_rn(b - __half2float(bh)));
  }
  uint4 *dst = reinterpret_cast<uint4 *>(hl + (row * C::kCPS + zq) * kRowBytes);
  dst[0] = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  dst[1] = make_uint4(hw[4], hw[5], hw[6], hw[7]);
  dst[2] = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  dst[3] = make_uint4(lw[4], lw[5], lw[6], lw[7]);
  if (zq == 0) {
    box_em[row] = make_int2(m > 0.f ? e : kNoExp, __float_as_int(sum));  // one 8-byte read for k_col_exp
  }
}

// Per tile column (parent): the column scale exponent (the smallest row
// exponent of its block, i.e. the scale of its largest |value|) and the total
// mass of each child's interaction zone (block total minus the child's 3^3
// near slots). A block of 8 warps takes 32 columns, lane = column (the rows
// of a slot are read coalesced), warp w the slots w, w + 8, ... with
// compensated FP32 sums (s, c); the 8 warps' sums of a column are then added
// in warp order with error-free two-sums (deterministic), so no FP64
// instruction is needed (each would hold the FP64 pipe for a whole warp).
__device__ __forceinline__ void kahan_add_f(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// (s, e) += (s2, e2), the value held being s + e with e small
__device__ __forceinline__ void two_sum_add(float &s, float &e, float s2, float e2) {
  const float t = s + s2;
  const float bp = t - s;
  e = e + e2 + ((s - (t - bp)) + (s2 - bp));
  s = t;
}

constexpr int kColWarps = 8;
__global__ void __launch_bounds__(32 * kColWarps) k_col_exp(int64_t ntiles, int kTileN, const int *__restrict__ rows,
                                                           const int2 *__restrict__ box_em,
                                                           int *__restrict__ col_exp,
                                                           float *__restrict__ zone_mass) {
  __shared__ float sh_s[kColWarps][9][32], sh_e[kColWarps][9][32];
  __shared__ int sh_x[kColWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;  // this lane's column
  const bool live = i < ntiles * kTileN;
  int e = kNoExp;
  float ts = 0.f, tc = 0.f, ns[8], nc[8];
#pragma unroll
  for (int o = 0; o < 8; ++o) ns[o] = nc[o] = 0.f;
  if (live) {
    const int *rr = rows + (i / kTileN) * kSlots * kTileN + (i % kTileN);
#pragma unroll 3
    for (int s = w; s < kSlots; s += kColWarps) {
      const int row = __ldg(rr + (int64_t)s * kTileN);
      if (row < 0) continue;
      const int2 em = __ldg(box_em + row);
      e = min(e, em.x);
      const float m = __int_as_float(em.y);
      kahan_add_f(ts, tc, m);
      // child o = ox + 2 oy + 4 oz is near slot s iff each coordinate lies in
      // [1 + o_axis, 3 + o_axis]: per axis the children (bit 0: o_axis = 0,
      // bit 1: o_axis = 1) are 0, 1, 3, 3, 2, 0 for coordinates 0 .. 5
      const unsigned mx = (0x2F4u >> (2 * (s % 6))) & 3u, my = (0x2F4u >> (2 * ((s / 6) % 6))) & 3u,
                     mz = (0x2F4u >> (2 * (s / 36))) & 3u;
      if (mx && my && mz) {
#pragma unroll
        for (int o = 0; o < 8; ++o)
          if ((mx >> (o & 1)) & (my >> ((o >> 1) & 1)) & (mz >> (o >> 2)) & 1u) kahan_add_f(ns[o], nc[o], m);
      }
    }
  }
  // Kahan's (s, c) holds s - c
  sh_s[w][8][lane] = ts;
  sh_e[w][8][lane] = -tc;
#pragma unroll
  for (int o = 0; o < 8; ++o) {
    sh_s[w][o][lane] = ns[o];
    sh_e[w][o][lane] = -nc[o];
  }
  sh_x[w][lane] = e;
  __syncthreads();
  if (w == 0 && live) {
    float s9[9], e9[9];
    int x = kNoExp;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      s9[q] = sh_s[0][q][lane];
      e9[q] = sh_e[0][q][lane];
    }
    for (int v = 0; v < kColWarps; ++v) {
      x = min(x, sh_x[v][lane]);
      if (v == 0) continue;
#pragma unroll
      for (int q = 0; q < 9; ++q) two_sum_add(s9[q], e9[q], sh_s[v][q][lane], sh_e[v][q][lane]);
    }
    col_exp[i] = x == kNoExp ? 0 : x;
#pragma unroll
    for (int o = 0; o < 8; ++o) zone_mass[i * 8 + o] = (s9[8] - s9[o]) + (e9[8] - e9[o]);
  }
}

template <int NG, int TN>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1) k_m2l_tc(const __grid_constant__ Params pr) {
  using C = Cfg<NG, TN>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  // full: this CTA's stage landed; pfull (leader): the peer's stage landed;
  // empty: the pair's MMAs are done with the stage; accf[x] / acce[x]:
  // accumulator buffer x filled by the MMAs / drained by both CTAs (leader)
  __shared__ uint64_t full[C::kStages], pfull[C::kStages], empty[C::kStages], accf[2], acce[2], never;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long lim = pr.wait_limit;
  const uint32_t rank = cluster_rank();  // 0: leader (issues the MMAs), 1: peer
  // this CTA's tile and row block q (rows 128 q ... of W); the two CTAs of a
  // cluster take the row blocks 2k and 2k + 1 of one tile (rank = q & 1)
  int64_t tile;
  int q;
  if (pr.qmajor) {
    const int64_t cid = blockIdx.x >> 1;
    tile = cid % pr.ntiles;
    q = 2 * (int)(cid / pr.ntiles) + (int)(blockIdx.x & 1);
  } else {
    tile = blockIdx.x / C::kQuarters;
    q = (int)(blockIdx.x % C::kQuarters);
  }
  int lev = 2;
  while (lev + 1 < pr.nlev && pr.tile_off[lev + 1] <= tile) ++lev;

  if (tid == 0) {
    for (int s = 0; s < C::kStages; ++s) {
      bar_init(&full[s], 1 + 32 * kGatherWarps);  // the W copy (with its byte count), then each gather thread
      bar_init(&pfull[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int x = 0; x < 2; ++x) {
      bar_init(&accf[x], 1);
      bar_init(&acce[x], 16);  // the 8 drain warps of each CTA
    }
    bar_init(&never, 1);  // nothing arrives here (the stall test hook)
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cluster_sync();  // both CTAs running, their barriers initialised
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // tensor memory allocated in both CTAs before the first MMA
  tc_fence_after();
  const uint32_t tbase = tmem_base;  // block b accumulates in columns kAccStride (b & 1) ...

  if (warp < kProdWarp0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsCtl));
    if (warp == 0) {
      // W tiles: the 4 K-chunks of a stage are one contiguous 32 KB block
      if (lane == 0) {
        const unsigned char *src = pr.w + (int64_t)(lev - 2) * C::kLevelBytes + (int64_t)q * C::kChunks * kABytes;
        bool ok = true;
        for (int u = 0; u < C::kSlotUses; ++u) {
          const int st = u % C::kStages;
          if (!bar_wait(&empty[st], ((u / C::kStages) & 1) ^ 1, lim)) {
            failed = 1;
            ok = false;
            break;
          }
          bar_expect(&full[st], C::kStageABytes);
          bulk_load(sm + st * C::kStageBytes, src + (int64_t)u * C::kStageABytes, C::kStageABytes, &full[st]);
        }
        // the releases of the last stages are the leader's final arrivals on
        // this CTA's barriers: wait for them before the CTA may leave
        for (int u = C::kSlotUses; ok && u < C::kSlotUses + C::kStages; ++u)
          if (!bar_wait(&empty[u % C::kStages], ((u / C::kStages) & 1) ^ 1, lim)) {
            failed = 1;
            ok = false;
          }
      }
    } else if (warp == 1 && rank == 0) {
      if (lane == 0) {
        // test hook: a wait that runs out; the CTAs give up and report it
        const bool stalled = pr.stall && !bar_wait(&never, 0, lim);
        if (stalled) failed = 1;
        for (int u = 0; !stalled && u < C::kSlotUses; ++u) {
          const int st = u % C::kStages;
          const int c0 = u * C::kStageChunks;  // first K-chunk of the stage
          const int b = c0 / C::kBlockChunks, x = b & 1;
          const bool first = (c0 % C::kBlockChunks) == 0;
          if (first && b >= 2) {
            // buffer x was last filled by block b - 2: wait for both CTAs' drains
            if (!bar_wait_cl(&acce[x], ((b >> 1) - 1) & 1, lim)) {
              failed = 1;
              break;
            }
            tc_fence_after();
          }
          if (!bar_wait(&full[st], (u / C::kStages) & 1, lim) || !bar_wait_cl(&pfull[st], (u / C::kStages) & 1, lim)) {
            failed = 1;
            break;
          }
          fence_async_smem();  // this CTA's gathered tiles were written by cp.async
          tc_fence_after();
          // rows hold 16 hi then 16 lo values: hi*hi, hi*lo, lo*hi; the same
          // offsets in the peer CTA hold its 128 rows of W and 128 parents
          const uint32_t sa = su32(sm + st * C::kStageBytes), sb = sa + C::kStageABytes;
          const uint32_t tacc = tbase + (uint32_t)C::kAccStride * (uint32_t)x;
#pragma unroll
          for (int k = 0; k < C::kStageChunks; ++k) {
            const uint32_t a = sa + k * kABytes, bb = sb + k * C::kBBytes;
            const uint64_t ah = sdesc(a), al = sdesc(a + 32), bh = sdesc(bb), bl = sdesc(bb + 32);
            mma(tacc, ah, bh, C::kIdesc, !(first && k == 0));
            mma(tacc, ah, bl, C::kIdesc, 1);
            mma(tacc, al, bh, C::kIdesc, 1);
          }
          mma_commit(&empty[st]);
          if ((c0 + C::kStageChunks) % C::kBlockChunks == 0) mma_commit(&accf[x]);
        }
      }
    } else if (warp >= 2 && rank == 1) {
      // peer: relay each landed stage to the leader (warp 2 the even stage
      // uses, warp 3 the odd ones, so each has two stages' time per arrival)
      if (lane == 0) {
        for (int u = warp - 2; u < C::kSlotUses; u += 2) {
          const int st = u % C::kStages;
          if (!bar_wait(&full[st], (u / C::kStages) & 1, lim)) {
            failed = 1;
            break;
          }
          fence_async_smem();  // the gathered tiles were written by cp.async
          bar_arrive_remote(&pfull[st], 0);
        }
      }
    }
  } else if (warp < kEpiWarp0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegsGather));
    // Gather warp g fills the B tiles of K-chunks g, g + 4, ... of every stage
    // use u (chunk c = kStageChunks u + g + 4 i: node chunk j of source slot s,
    // nodes 16 j ... of the slot's gridlet) with this CTA's kHalfN parents
    // (kHalfN rank ...): 64 bytes each, 4 lanes per parent (one 16-byte piece
    // each), parents 8 m + lane / 4. Each thread's copies arrive on the
    // stage's full barrier when they land (cp.async.mbarrier.arrive.noinc);
    // the thread that consumes the stage (the leader's MMA thread, the peer's
    // relay) makes them visible to the tensor core's proxy with one fence per
    // stage, much cheaper there than a fence per gathering warp after its
    // copies. When the warp's next chunk lies in the next slot, that slot's row
    // indices are loaded while the current chunk is copied.
    const int g = warp - kProdWarp0, sub = lane & 3, grp = lane >> 2;
    const int *rp = pr.rows + tile * kSlots * C::kTileN + (int)rank * C::kHalfN + grp;
    // sw64 position of parent 8 m + grp, piece sub: 512 m + this lane's offset
    const uint32_t lane_off = (uint32_t)(grp * 64 + ((sub ^ ((grp >> 1) & 3)) << 4));
    const uint32_t bsh = su32(sm + C::kStageABytes + g * C::kBBytes) + lane_off;
    const unsigned char *hsub = pr.hl + 16 * sub;
    constexpr int kPer = C::kHalfN / 8;
    constexpr int kGPer = C::kStageChunks / kGatherWarps;  // this warp's chunks per stage
    // at Ng = 4 a slot is 4 chunks: the warp's next chunk is always in the next slot
    constexpr bool kAlwaysNext = C::kCPS == kGatherWarps;
    int rows[kPer], next[kPer];
    {
      const int s0 = g / C::kCPS;
#pragma unroll
      for (int m = 0; m < kPer; ++m) rows[m] = __ldg(rp + s0 * C::kTileN + 8 * m);
    }
    for (int u = 0; u < C::kSlotUses; ++u) {
      const int st = u % C::kStages;
      int ok = 1;
      if (lane == 0) ok = bar_wait(&empty[st], ((u / C::kStages) & 1) ^ 1, lim);
      if (!__shfl_sync(0xffffffffu, ok, 0)) {
        failed = 1;
        break;
      }
#pragma unroll
      for (int ch = 0; ch < kGPer; ++ch) {
        const int c = u * C::kStageChunks + g + ch * kGatherWarps, s = c / C::kCPS, j = c - s * C::kCPS;
        const int sn = (c + kGatherWarps) / C::kCPS;  // slot of this warp's next chunk (s or s + 1)
        if (kAlwaysNext || sn != s) {
#pragma unroll
          for (int m = 0; m < kPer; ++m) next[m] = sn < kSlots ? __ldg(rp + sn * C::kTileN + 8 * m) : -1;
        }
        const uint32_t dst = bsh + st * C::kStageBytes + ch * kGatherWarps * C::kBBytes;
        const unsigned char *hj = hsub + j * kRowBytes;
#pragma unroll
        for (int m = 0; m < kPer; ++m) {
          const int row = rows[m];
          cp16(dst + m * 512, hj + (int64_t)(row >= 0 ? row : 0) * C::kCPS * kRowBytes, row >= 0 ? 16u : 0u);
        }
        if (kAlwaysNext || sn != s) {
#pragma unroll
          for (int m = 0; m < kPer; ++m) rows[m] = next[m];
        }
      }
      asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(su32(&full[st])) : "memory");
    }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegsHigh));
    // drain: total += block accumulator (registers); after the last block
    // write the values. Warp w reads TMEM lanes 32 (w mod 4) ...
    const int lq = warp & 3, half = (warp - kEpiWarp0) >> 2;
    const int r = lq * 32 + lane;                 // row of this thread in the CTA's block
    const int R = q * kRows + r;                  // row of W: child o, node
    const bool real_row = C::kRowsReal % kRows == 0 || R < C::kRowsReal;  // no padding rows at Ng = 4
    const int o = real_row ? R / C::kM3 : 0, node = R - o * C::kM3;
    const uint32_t lane_off = (uint32_t)(lq * 32) << 16;
    const int e_row = __ldg(pr.w_exp + (lev - 2) * (C::kQuarters * kRows) + q * kRows + r);
    // running totals of this thread's kCols columns: FP32, or compensated
    // (the exact rounding error of every addition to tot accumulates in a
    // bf16 compensation term, two columns per register: the total is
    // tot + compensation, several bits beyond FP32 for a few registers)
    constexpr int kCols = C::kCols, kG = C::kColGroup, kGroups = kCols / kG;
    float tot[kCols];
    uint32_t comp[C::kDfTotals ? kCols / 2 : 1];
    if constexpr (C::kDfTotals) {
#pragma unroll
      for (int j = 0; j < kCols; ++j) tot[j] = 0.f;  // two-sums into zero are exact
#pragma unroll
      for (int j = 0; j < kCols / 2; ++j) comp[j] = 0u;
    }
    bool ok = true;
#pragma unroll 1
    for (int b = 0; b < C::kBlocks; ++b) {
      const int x = b & 1;
      if (!__all_sync(0xffffffffu, bar_wait_cl(&accf[x], (b >> 1) & 1, lim))) {
        failed = 1;
        ok = false;
        break;
      }
      tc_fence_after();
      if constexpr (C::kDfTotals) {
        // 8 columns per load: the double-float totals leave few registers
#pragma unroll
        for (int cc = 0; cc < kCols / 8; ++cc) {
          uint32_t a[8];
          tmem_ld8(tbase + (uint32_t)C::kAccStride * (uint32_t)x + lane_off + half * kCols + cc * 8, a);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            float e[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const float v = __uint_as_float(a[j + h]);
              const float s0 = tot[cc * 8 + j + h], t = s0 + v, bp = t - s0;
              e[h] = (s0 - (t - bp)) + (v - bp);  // exact rounding error of s0 + v
              tot[cc * 8 + j + h] = t;
            }
            uint32_t &cw = comp[(cc * 8 + j) / 2];
            const __nv_bfloat162 nc = __floats2bfloat162_rn(__uint_as_float(cw << 16) + e[0],
                                                            __uint_as_float(cw & 0xffff0000u) + e[1]);
            cw = *reinterpret_cast<const uint32_t *>(&nc);
          }
        }
      } else {
#pragma unroll
        for (int cc = 0; cc < kGroups; ++cc) {
          uint32_t a[kG];
          const uint32_t ta = tbase + (uint32_t)C::kAccStride * (uint32_t)x + lane_off + half * kCols + cc * kG;
          if constexpr (kG == 32) tmem_ld32(ta, a);
          else if constexpr (kG == 16) tmem_ld16(ta, a);
          else tmem_ld8(ta, a);
          tmem_wait_ld();
          if (b == 0) {
#pragma unroll
            for (int j = 0; j < kG; ++j) tot[cc * kG + j] = __uint_as_float(a[j]);
          } else {
#pragma unroll
            for (int j = 0; j < kG; ++j) tot[cc * kG + j] = __uint_as_float(a[j]) + tot[cc * kG + j];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (rank == 0) bar_arrive(&acce[x]);
        else bar_arrive_remote(&acce[x], 0);
      }
    }
    if constexpr (C::kDfTotals) {
#pragma unroll
      for (int j = 0; j < kCols / 2; ++j) {  // the compensated totals, rounded once
        tot[2 * j] += __uint_as_float(comp[j] << 16);
        tot[2 * j + 1] += __uint_as_float(comp[j] & 0xffff0000u);
      }
    }
    if (ok && real_row) {
#pragma unroll
      for (int cc = 0; cc < kGroups; ++cc) {
        const int col = half * kCols + cc * kG;
        const int *tg = pr.tgt + (tile * C::kTileN + col) * 8 + o;
        const int *ce = pr.col_exp + tile * C::kTileN + col;
#pragma unroll
        for (int j = 0; j < kG; ++j) {
          const int t_idx = __ldg(tg + j * 8);
          if (t_idx >= 0) {
            const float v = (tot[cc * kG + j] * pow2f(-e_row)) * pow2f(-__ldg(ce + j));
            if (node == 0) {
              pr.outc[t_idx] = (float)((double)v + pr.mean[lev][o] * (double)__ldg(pr.zone_mass + (tile * C::kTileN + col + j) * 8 + o));
              pr.out[(int64_t)t_idx * C::kM3] = 0.f;
            } else {
              pr.out[(int64_t)t_idx * C::kM3 + node] = v;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no arrivals on, or reads of, the other CTA after this
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
  }
  if (tid == 0 && failed) atomicOr(pr.err, kErrTimeout);
}

}  // namespace tc

bool use_tc_m2l(const hpm_plan_s *pl) {
  return (pl->ng == 4 || pl->ng == 6) &&
         !(pl->opts.flags &
           (HPM_FLAG_GENERIC_M2L | HPM_FLAG_XTRANSFORM_M2L | HPM_FLAG_FFT_M2L | HPM_FLAG_EXTENDED_GRIDLET));
}

namespace {

template <int NG>
hpm_status tc_precompute_ng(hpm_plan_s *pl, cudaStream_t st) {
  using C = tc::Cfg<NG>;
  const int D = pl->max_depth;
  HPM_TRY(pl->tc_w.ensure((size_t)C::kLevelBytes * (D - 1), st));
  HPM_TRY(pl->tc_wexp.ensure(sizeof(int) * C::kQuarters * tc::kRows * (D - 1), st));
  HPM_CUDA(cudaMemsetAsync(pl->tc_wexp.p, 0, sizeof(int) * C::kQuarters * tc::kRows * (D - 1), st));
  HPM_TRY(pl->tc_mean.ensure(sizeof(double) * 8 * (D + 1), st));
  // m_o: mean of -g(h |y_{o,0} - y_{s,j}|) over the zone's 189 slots x Ng^3 nodes
  std::vector<double> mean(8 * (D + 1), 0.0);
  for (int l = 2; l <= D; ++l) {
    const double *gl = pl->glat_host.data() + pl->glat_stride * l;
    for (int o = 0; o < 8; ++o) {
      const int px = 2 + (o & 1), py = 2 + ((o >> 1) & 1), pz = 2 + (o >> 2);
      double sum = 0.0;
      int64_t cnt = 0;
      for (int s = 0; s < tc::kSlots; ++s) {
        const int sx = s % 6, sy = (s / 6) % 6, sz = s / 36;
        if (std::max(std::abs(sx - px), std::max(std::abs(sy - py), std::abs(sz - pz))) <= 1) continue;
        for (int j = 0; j < C::kM3; ++j) {
          const int dx = NG * px - (NG * sx + j % NG), dy = NG * py - (NG * sy + (j / NG) % NG),
                    dz = NG * pz - (NG * sz + j / (NG * NG));
          sum += -gl[dx * dx + dy * dy + dz * dz];
          ++cnt;
        }
      }
      mean[8 * l + o] = sum / (double)cnt;
    }
  }
  pl->tc_mean_host = mean;
  HPM_CUDA(cudaMemcpyAsync(pl->tc_mean.p, mean.data(), sizeof(double) * mean.size(), cudaMemcpyHostToDevice, st));
  const int64_t nthr = (int64_t)C::kQuarters * C::kChunks * tc::kRows;
  const unsigned nblk = (unsigned)((nthr + 255) / 256);
  int *rowmax = nullptr;
  HPM_TRY(lib_malloc_async((void **)&rowmax, sizeof(int) * C::kQuarters * tc::kRows, st));
  for (int l = 2; l <= D; ++l) {
    const double *gl = pl->glat.as<double>() + pl->glat_stride * l;
    const double *mean_l = pl->tc_mean.as<double>() + 8 * l;
    int *wexp = pl->tc_wexp.as<int>() + C::kQuarters * tc::kRows * (l - 2);
    HPM_CUDA(cudaMemsetAsync(rowmax, 0, sizeof(int) * C::kQuarters * tc::kRows, st));
    tc::k_w_rowmax<NG><<<nblk, 256, 0, st>>>(gl, mean_l, rowmax);
    HPM_LAUNCHED((int64_t *)nullptr);
    tc::k_w_table<NG><<<nblk, 256, 0, st>>>(gl, mean_l, rowmax,
                                            pl->tc_w.as<unsigned char>() + C::kLevelBytes * (l - 2), wexp);
    HPM_LAUNCHED((int64_t *)nullptr);
  }
  HPM_CUDA(cudaFreeAsync(rowmax, st));
  // the mean vector is host memory the copy above reads
  HPM_CUDA(cudaStreamSynchronize(st));
  return HPM_OK;
}

template <int NG, int TN>
hpm_status launch_m2l_tc_ng(hpm_plan_s *pl, cudaStream_t st, int64_t *launches) {
  using C = tc::Cfg<NG, TN>;
  const int64_t off2 = pl->lvl_off[2], nrow = pl->nbox - off2;
  if (nrow <= 0) return HPM_OK;
  HPM_TRY(pl->s.grid_hl.ensure((size_t)nrow * C::kCPS * tc::kRowBytes, st));
  HPM_TRY(pl->s.box_em.ensure(sizeof(int2) * nrow, st));
  HPM_TRY(pl->s.col_exp.ensure(sizeof(int) * pl->tc_ntiles * C::kTileN, st));
  HPM_TRY(pl->s.zone_mass.ensure(sizeof(float) * pl->tc_ntiles * C::kTileN * 8, st));
  tc::RowLevels rl{};
  rl.nlev = pl->max_depth + 1;
  for (int l = 0; l <= pl->max_depth + 1; ++l) rl.off[l] = pl->lvl_off[l];
  rl.off2 = off2;
  // the per-(problem, level) maxima were taken by the P2G and child-to-parent
  // kernels as they wrote the rows (s.level_amax)
  constexpr int kL = C::kCPS <= 4 ? 4 : (C::kCPS <= 8 ? 8 : (C::kCPS <= 16 ? 16 : 32));
  tc::k_split<NG><<<(unsigned)((kL * nrow + 255) / 256), 256, 0, st>>>(
      nrow, pl->s.grid.as<float>(), pl->t.box_key.as<uint64_t>(), rl, pl->s.level_amax.as<int>(),
      pl->s.grid_hl.as<unsigned char>(), pl->s.box_em.as<int2>());
  HPM_LAUNCHED(launches);
  tc::k_col_exp<<<(unsigned)((pl->tc_ntiles * C::kTileN + 31) / 32), 32 * tc::kColWarps, 0, st>>>(
      pl->tc_ntiles, C::kTileN, pl->t.tc_rows.as<int>(), pl->s.box_em.as<int2>(),
      pl->s.col_exp.as<int>(), pl->s.zone_mass.as<float>());
  HPM_LAUNCHED(launches);
  tc::Params p{};
  p.w = pl->tc_w.as<unsigned char>();
  p.w_exp = pl->tc_wexp.as<int>();
  p.col_exp = pl->s.col_exp.as<int>();
  p.hl = pl->s.grid_hl.as<unsigned char>();
  p.zone_mass = pl->s.zone_mass.as<float>();
  p.rows = pl->t.tc_rows.as<int>();
  p.tgt = pl->t.tc_tgt.as<int>();
  for (int l = 0; l <= kMaxDepth + 1; ++l) p.tile_off[l] = l < (int)pl->tc_tile_off.size() ? pl->tc_tile_off[l] : 0;
  p.ntiles = pl->tc_ntiles;
  p.qmajor = m2l_block_order(pl) == 2 ? 1 : 0;
  p.nlev = pl->max_depth + 1;
  p.out = pl->s.m2l_raw.as<float>();
  p.outc = pl->s.m2lc.as<float>();
  p.err = pl->t.err.as<int>() + 1;  // the solves' error word
  p.wait_limit = pl->test_wait_limit > 0 ? pl->test_wait_limit : (1ll << 32);
  p.stall = pl->test_stall;
  for (int l = 0; l <= kMaxDepth && 8 * l + 7 < (int)pl->tc_mean_host.size(); ++l)
    for (int o = 0; o < 8; ++o) p.mean[l][o] = pl->tc_mean_host[8 * l + o];
  static DeviceCache attr_cache;
  int attr_ok = 0;
  HPM_TRY(device_cached(attr_cache, [](int *v) -> hpm_status {
    HPM_CUDA(cudaFuncSetAttribute(tc::k_m2l_tc<NG, TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmem));
    // The drain warps raise their register count to kRegsHigh with registers
    // the other warpgroups give back; that only adds up if the kernel was
    // compiled with kLaunchRegs per thread. Never launch it otherwise.
    cudaFuncAttributes fa{};
    HPM_CUDA(cudaFuncGetAttributes(&fa, tc::k_m2l_tc<NG, TN>));
    if (fa.numRegs != tc::kLaunchRegs)
      fprintf(stderr, "hpm: k_m2l_tc<%d, %d> compiled with %d registers per thread, expected %d\n", NG, TN,
              fa.numRegs, tc::kLaunchRegs);
    *v = fa.numRegs == tc::kLaunchRegs ? 1 : 0;
    return HPM_OK;
  }, &attr_ok));
  if (!attr_ok) return HPM_ERR_UNSUPPORTED;
  const int64_t grid = pl->tc_ntiles * C::kQuarters;
  if (pl->events_ready) cudaEventRecord(pl->ev[10], st);
  tc::k_m2l_tc<NG, TN><<<(unsigned)grid, tc::kThreads, C::kSmem, st>>>(p);
  HPM_LAUNCHED(launches);
  if (pl->events_ready) cudaEventRecord(pl->ev[11], st);
  pl->stats.m2l_parents = pl->npar;
  return HPM_OK;
}

}  // namespace

int m2l_tile_parents(const hpm_plan_s *pl) {
  if (pl->ng != 4) return tc::Cfg<6>::kTileN;
  const int t = pl->tuning.m2l_tile_parents;
  return t == 224 || t == 208 || t == 192 ? t : 256;
}

int m2l_block_order(const hpm_plan_s *pl) {
  const int o = pl->tuning.m2l_block_order;
  return o == 1 || o == 2 ? o : 1;  // tile-major unless tuned otherwise
}

hpm_status tc_precompute(hpm_plan_s *pl, cudaStream_t st) {
  if (!use_tc_m2l(pl) || pl->max_depth < 2) return HPM_OK;
  return pl->ng == 6 ? tc_precompute_ng<6>(pl, st) : tc_precompute_ng<4>(pl, st);
}

hpm_status tc_build_tiles(hpm_plan_s *pl, const std::vector<int64_t> &par_per_level, cudaStream_t st,
                          int64_t *launches) {
  pl->tc_ntiles = 0;
  pl->tc_tile_off.assign(kMaxDepth + 2, 0);
  if (!use_tc_m2l(pl)) return HPM_OK;
  const int D = pl->max_depth;
  const int tile_n = m2l_tile_parents(pl);  // the solve launches the kernel of this width
  pl->tc_tile_n = tile_n;
  tc::TileLevels tl{};
  tl.nlev = D + 1;
  int64_t tiles = 0, pars = 0;
  for (int l = 0; l <= D + 1; ++l) {
    tl.tile_off[l] = tiles;
    tl.par_off[l] = pars;
    pl->tc_tile_off[l] = tiles;
    if (l >= 2 && l <= D) {
      const int64_t np = par_per_level[l - 1];  // parents of level-l targets sit at level l - 1
      tiles += (np + tile_n - 1) / tile_n;
      pars += np;
    }
  }
  if (pars != pl->npar) return HPM_ERR_INVALID_ARG;
  pl->tc_ntiles = tiles;
  if (!tiles) return HPM_OK;
  const int64_t off2 = pl->lvl_off[2];
  HPM_TRY(pl->t.tc_rows.ensure(sizeof(int) * tiles * tc::kSlots * tile_n, st));
  HPM_TRY(pl->t.tc_tgt.ensure(sizeof(int) * tiles * tile_n * 8, st));
  const int64_t nthr = tiles * tile_n;
  tc::k_tiles<<<(unsigned)((nthr + 255) / 256), 256, 0, st>>>(
      tiles, tile_n, tl, pl->t.par_box.as<int>(), pl->t.box_nb.as<int>(), pl->t.box_child.as<int>(),
      pl->t.box_tgt.as<int>(), off2, pl->t.tc_rows.as<int>(), pl->t.tc_tgt.as<int>());
  HPM_LAUNCHED(launches);
  return HPM_OK;
}

hpm_status launch_m2l_tc(hpm_plan_s *pl, cudaStream_t st, int64_t *launches) {
  if (!pl->tc_ntiles) return HPM_OK;
  if (pl->ng == 6) return launch_m2l_tc_ng<6, 128>(pl, st, launches);
  switch (pl->tc_tile_n) {  // the width the tiles were built with
    case 224: return launch_m2l_tc_ng<4, 224>(pl, st, launches);
    case 208: return launch_m2l_tc_ng<4, 208>(pl, st, launches);
    case 192: return launch_m2l_tc_ng<4, 192>(pl, st, launches);
    default: return launch_m2l_tc_ng<4, 256>(pl, st, launches);
  }
}

}  // namespace hpm
