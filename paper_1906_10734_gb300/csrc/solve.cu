// Solve stages other than the source-to-target convolution:
//   gather      sorted particle copies (FP64 for the gridlet weights, FP32
//               hi/lo for the near field)
//   P2G         effective masses of leaves and virtual boxes (Sec. 2.2)
//   M2M         child-to-parent with the separable T^C (Sec. 2.3)
//   L2L         parent-to-child, Phi^C_p = Phi^P((a^C + x_p)/2) (Sec. 2.4)
//   G2P         interpolant of Eq. phix and its gradient at the particles
//   P2P         near zone by direct summation with Kahan-compensated FP32
//   Green       FP64 transform of the exact Green function (Sec. 2.1, Eq. gf)
#include <cmath>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

// Sorted particle: FP64 position and mass.

constexpr int kThreads = 256;
constexpr int kWarpsPerBlock = kThreads / 32;

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }
inline unsigned warp_blocks(int64_t n) { return (unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock); }

// M2M and L2L hold three Ng^3 buffers per warp: 4 warps per block keep the
// static shared memory under 48 KB for Ng = 8.
constexpr int kGThreads = 128;
constexpr int kGWarps = kGThreads / 32;
inline unsigned gwarp_blocks(int64_t n) { return (unsigned)((n + kGWarps - 1) / kGWarps); }

struct LevelTable {
  int64_t off[kMaxDepth + 3];
  int nlev;
};

__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x1fffffull;
  return (uint32_t)x;
}

__device__ __forceinline__ int level_of(const LevelTable &lt, int64_t box) {
  int l = 0;
  while (l + 1 < lt.nlev && lt.off[l + 1] <= box) ++l;
  return l;
}

// ---------------------------------------------------------------------------
// IEEE 754 conversions between binary32 and binary64 by bit manipulation on
// the integer units (the FP64 pipe of this GPU issues about 2 operations per
// SM-cycle, conversions included): float -> double is exact, the exponent
// re-biased by 1023 - 127 = 896 and the 23-bit fraction shifted up by 29;
// double -> float rounds to nearest, ties to even, on the 29 dropped fraction
// bits (a carry out of the fraction steps the exponent, which is the IEEE
// result, up to infinity). Zeros are signed zeros; subnormals, infinities,
// NaNs and doubles outside the float normal range take the hardware
// conversion. Both give the hardware's bits.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f), a = b & 0x7FFFFFFFu;
  if (a - 0x00800000u >= 0x7F000000u) return a ? (double)f : __hiloint2double((int)(b & 0x80000000u), 0);
  return __hiloint2double((int)((b & 0x80000000u) | ((a >> 3) + 0x38000000u)), (int)(b << 29));
}
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ha = hi & 0x7FFFFFFFu;
  // biased double exponent 897 .. 1150: the float normal range
  if (ha - 0x38100000u >= 0x0FE00000u) return (ha | lo) ? (float)x : __uint_as_float(hi & 0x80000000u);
  unsigned r = ((ha - 0x38000000u) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1FFFFFFFu;
  r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;
  return __uint_as_float((hi & 0x80000000u) | r);
}

// Self-check of the two conversions against the hardware's (NaNs compare by
// class): the number of inputs whose bits differ.
__global__ void k_check_conversions(const double *__restrict__ d, int64_t nd, const float *__restrict__ f,
                                    int64_t nf, unsigned long long *__restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned c = 0;
  if (i < nd) {
    const float a = f64_to_f32_rn(d[i]), h = (float)d[i];
    c += (__float_as_uint(a) != __float_as_uint(h)) && !(isnan(a) && isnan(h));
  }
  if (i < nf) {
    const double a = f32_to_f64(f[i]), h = (double)f[i];
    c += (__double_as_longlong(a) != __double_as_longlong(h)) && !(isnan(a) && isnan(h));
  }
  if (c) atomicAdd(bad, (unsigned long long)c);
}

template <bool kUnit>
__global__ void k_gather(int64_t n, const uint32_t *__restrict__ perm, const double *__restrict__ pos,
                         const double *__restrict__ mass, double ox, double oy, double oz, double inv_side,
                         float4 *__restrict__ hi, float4 *__restrict__ lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t p = perm[i];
  const double x = pos[3 * (int64_t)p], y = pos[3 * (int64_t)p + 1], z = pos[3 * (int64_t)p + 2];
  // position in the unit cube of the domain, u = (x - o) / S, as an
  // unevaluated sum hi + lo of two floats: a cell-relative coordinate
  // u 2^l - c is then exact in FP32 up to one rounding, and differences of
  // nearby particles keep FP32 precision relative to themselves. kUnit: the
  // domain is the unit cube at the origin, u = x (two FP64 operations fewer
  // per axis on this GPU's narrow FP64 pipe)
  const double ux = kUnit ? x : (x - ox) * inv_side, uy = kUnit ? y : (y - oy) * inv_side,
               uz = kUnit ? z : (z - oz) * inv_side;
  // (the conversions on the integer units: this kernel is otherwise bound by
  // the FP64 pipe's conversions)
  const float hx = f64_to_f32_rn(ux), hy = f64_to_f32_rn(uy), hz = f64_to_f32_rn(uz);
  hi[i] = make_float4(hx, hy, hz, f64_to_f32_rn(mass[p]));
  lo[i] = make_float4(f64_to_f32_rn(ux - f32_to_f64(hx)), f64_to_f32_rn(uy - f32_to_f64(hy)),
                      f64_to_f32_rn(uz - f32_to_f64(hz)), 0.f);
}

// The same in FP64 (exact up to one FP64 rounding): the input of the
// moment-matching weights.
__device__ __forceinline__ double cell_coord_d(float h, float lo, float scale, float c) {
  return (double)fmaf(h, scale, -c) + (double)lo * (double)scale;
}

// Cell-relative coordinate xi = u 2^l - c of a hi/lo unit-cube coordinate:
// h 2^l - c is exact (the two are within a factor two of each other away from
// the domain's first cell, where the error stays below 2^-26), so the result
// carries one FP32 rounding.
__device__ __forceinline__ float cell_coord(float h, float lo, float scale, float c) {
  return fmaf(h, scale, -c) + lo * scale;
}

// 1-D Lagrange weights on the gridlet nodes, FP64 (the moment-matching solve).
// With u = 2 Ng xi the nodes are the integers a_k = 2k + 1 - Ng, and
// ell_j = prod_{k != j} (u - a_k) / (a_j - a_k) is formed from prefix and
// suffix products of the differences.
// NG > 0 fixes the order at compile time (arrays stay in registers); NG = 0
// takes it from the table.
template <int NG>
__device__ __forceinline__ void lagrange_d(const GridletTables &tb, double xi, float *w) {
  const int ng = NG > 0 ? NG : tb.ng;
  const double u = xi * (double)(2 * ng);
  double d[kMaxNg], suf[kMaxNg];
#pragma unroll
  for (int k = 0; k < (NG > 0 ? NG : kMaxNg); ++k)
    if (k < ng) d[k] = u - (double)(2 * k + 1 - ng);
  suf[ng - 1] = 1.0;
#pragma unroll
  for (int k = (NG > 0 ? NG : kMaxNg) - 2; k >= 0; --k)
    if (k <= ng - 2) suf[k] = suf[k + 1] * d[k + 1];
  double pre = 1.0;
#pragma unroll
  for (int j = 0; j < (NG > 0 ? NG : kMaxNg); ++j)
    if (j < ng) {
      w[j] = (float)(tb.inv_den_u[j] * (pre * suf[j]));
      pre *= d[j];
    }
}

// Ng = 4 in closed form: with u = 8 xi = A + B (A, B floats whose sum is
// exact in FP64) and the nodes -3, -1, 1, 3, ell_0 = -(u+1)(u-1)(u-3)/48,
// ell_1 = (u+3)(u-1)(u-3)/16, ell_2 = -(u+3)(u+1)(u-3)/16 and
// ell_3 = (u+3)(u+1)(u-1)/48. The same FP64 products as the general form in
// fewer FP64 instructions; the factors 1/16 are powers of two and are applied
// after the rounding to FP32 (an exact scaling), so the weights are the same.
__device__ __forceinline__ void lagrange4_d(float A, float B, float *w) {
  const double u = (double)A + (double)B;
  const double d0 = u + 3.0, d1 = u + 1.0, d2 = u - 1.0, d3 = u - 3.0;
  const double e = d2 * d3, f = d0 * d1;
  // the products in FP64, rounded to FP32 once, then the denominators (+-16
  // exactly, +-48 to one more FP32 rounding)
  w[0] = (float)(d1 * e) * (-1.f / 48.f);
  w[1] = (float)(d0 * e) * 0.0625f;
  w[2] = (float)(f * d3) * -0.0625f;
  w[3] = (float)(f * d2) * (1.f / 48.f);
}

// The largest |effective mass| of a warp's gridlet (a = this lane's) into its
// (problem, level) slot: the per-level scale of the dense source-to-target
// kernel's FP16 planes, taken here as the rows are written (amax null on the
// other paths). Positive floats order as their bit patterns.
__device__ __forceinline__ void row_amax(int *amax, float a, const uint64_t *__restrict__ key, int64_t box,
                                         int level, int nlev) {
  const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(fabsf(a)));
  if (amax && (threadIdx.x & 31) == 0) atomicMax(amax + (int)(key[box] >> (3 * level)) * nlev + level, (int)m);
}

// Effective masses, M_p = sum_i m_i prod_d ell_{p_d}(xi_d) (Eq. mp in Lagrange
// form: sum_n B_pn t^n = ell_p(t)), for the boxes that are not expanded: each
// particle's finest box (an expanded box, internal or not, gets its gridlet
// from its children by the child-to-parent transform). A block takes 8 boxes;
// all its threads evaluate the FP64 weights of the (box, particle) pairs of
// those boxes, 256 pairs at a time, then warp w accumulates box w from shared
// memory.
template <int NG>
__global__ void __launch_bounds__(kThreads, NG == 4 ? 8 : 2) k_p2g(int64_t nbox, const int *__restrict__ list, LevelTable lt,
                                                  GridletTables tb, const uint64_t *__restrict__ key,
                                                  const int *__restrict__ beg, const int *__restrict__ end,
                                                  const float4 *__restrict__ uhi,
                                                  const float4 *__restrict__ ulo, int64_t off2,
                                                  float *__restrict__ grid, int *__restrict__ amax, int nlev) {
  // (weights of the block's pairs: Ng per axis; at Ng = 4 the smaller array and
  // 32 registers let 8 blocks share an SM, whose phases of FP64 weights and of
  // accumulation then overlap across blocks)
  __shared__ float ws[kThreads][3][NG > 0 ? NG : kMaxNg];
  __shared__ float ms[kThreads];
  __shared__ int off[kWarpsPerBlock + 1];
  __shared__ int bx[kWarpsPerBlock], bbeg[kWarpsPerBlock], blev[kWarpsPerBlock];
  __shared__ float bc[kWarpsPerBlock][3], bscale[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * kWarpsPerBlock;
  const int nb = (int)min((int64_t)kWarpsPerBlock, nbox - b0);
  // the block's (box, particle) pairs: the boxes' particle counts, prefixed
  int cnt = 0;
  if (threadIdx.x < nb) {
    const int box = list[b0 + threadIdx.x];
    cnt = end[box] - beg[box];
  }
  if (threadIdx.x < 32) {
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < kWarpsPerBlock; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if ((threadIdx.x & 31) >= o) inc += t;
    }
    if (threadIdx.x < nb) off[threadIdx.x + 1] = inc;
    if (threadIdx.x == 0) off[0] = 0;
  }
  if (threadIdx.x < nb) {
    const int box = list[b0 + threadIdx.x];
    const int l = level_of(lt, box);
    const uint64_t k = key[box] & ((1ull << (3 * l)) - 1ull);
    bx[threadIdx.x] = box;
    blev[threadIdx.x] = l;
    bbeg[threadIdx.x] = beg[box];
    bscale[threadIdx.x] = (float)(1u << l);
    bc[threadIdx.x][0] = (float)compact3(k) + 0.5f;
    bc[threadIdx.x][1] = (float)compact3(k >> 1) + 0.5f;
    bc[threadIdx.x][2] = (float)compact3(k >> 2) + 0.5f;
  }
  __syncthreads();
  const int ng = tb.ng, m3 = ng * ng * ng;
  constexpr int kR = NG > 0 ? (NG * NG * NG + 31) / 32 : 16;  // output rounds of 32 nodes
  float acc[kR];
#pragma unroll
  for (int r = 0; r < kR; ++r) acc[r] = 0.f;
  const int P0 = off[0], P1 = off[nb];
  for (int c0 = P0; c0 < P1; c0 += kThreads) {
    const int p = c0 + threadIdx.x;
    if (p < P1) {
      int lb = 0;
      while (lb + 1 < nb && off[lb + 1] <= p) ++lb;
      const int pi = bbeg[lb] + (p - off[lb]);
      const float4 h = uhi[pi], q = ulo[pi];
      const float sc = bscale[lb];
      if constexpr (NG == 4) {
        // u = 8 xi = 8 (h sc - c) + 8 lo sc: both parts exact in FP32 (powers of two)
        const float s8 = 8.f * sc;
        lagrange4_d(fmaf(h.x, s8, -8.f * bc[lb][0]), q.x * s8, ws[threadIdx.x][0]);
        lagrange4_d(fmaf(h.y, s8, -8.f * bc[lb][1]), q.y * s8, ws[threadIdx.x][1]);
        lagrange4_d(fmaf(h.z, s8, -8.f * bc[lb][2]), q.z * s8, ws[threadIdx.x][2]);
      } else {
        lagrange_d<NG>(tb, cell_coord_d(h.x, q.x, sc, bc[lb][0]), ws[threadIdx.x][0]);
        lagrange_d<NG>(tb, cell_coord_d(h.y, q.y, sc, bc[lb][1]), ws[threadIdx.x][1]);
        lagrange_d<NG>(tb, cell_coord_d(h.z, q.z, sc, bc[lb][2]), ws[threadIdx.x][2]);
      }
      ms[threadIdx.x] = h.w;
    }
    __syncthreads();
    if (w < nb) {
      const int jb = max(off[w], c0) - c0, je = min(off[w + 1], c0 + kThreads) - c0;
      if constexpr (NG == 4) {
        // nodes lane and lane + 32: the same x and y weights, z = lane/16 and 2 + lane/16
        const int px = lane & 3, py = (lane >> 2) & 3, pz = lane >> 4;
        float a0 = acc[0], a1 = acc[1];
        for (int j = jb; j < je; ++j) {
          const float t = ms[j] * ws[j][0][px] * ws[j][1][py];
          a0 = fmaf(t, ws[j][2][pz], a0);
          a1 = fmaf(t, ws[j][2][pz + 2], a1);
        }
        acc[0] = a0;
        acc[1] = a1;
      } else {
#pragma unroll
        for (int r = 0; r < kR; ++r) {
          const int pp = r * 32 + lane;
          if (pp >= m3) break;
          const int px = pp % ng, py = (pp / ng) % ng, pz = pp / (ng * ng);
          float s = acc[r];
          for (int j = jb; j < je; ++j) s += ms[j] * ws[j][0][px] * ws[j][1][py] * ws[j][2][pz];
          acc[r] = s;
        }
      }
    }
    __syncthreads();
  }
  if (w < nb) {
    float *out = grid + (int64_t)(bx[w] - off2) * m3;
    float a = 0.f;
#pragma unroll
    for (int r = 0; r < kR; ++r)
      if (r * 32 + lane < m3) {
        out[r * 32 + lane] = acc[r];
        a = fmaxf(a, fabsf(acc[r]));
      }
    row_amax(amax, a, key, bx[w], blev[w], nlev);
  }

}

// Separable application of a 1-D operator along one axis of an Ng^3 gridlet
// held in shared memory: dst[.., p_axis, ..] = sum_q op[p][q] src[.., q, ..]
// (or op[q][p] when transposed).
__device__ __forceinline__ void apply_axis(const float *__restrict__ op, bool transpose, int axis,
                                           int ng, const float *src, float *dst, bool accumulate) {
  const int lane = threadIdx.x & 31, m3 = ng * ng * ng;
  const int stride = axis == 0 ? 1 : (axis == 1 ? ng : ng * ng);
  for (int p = lane; p < m3; p += 32) {
    const int c = (p / stride) % ng;
    const int base = p - c * stride;
    float s = 0.f;
    for (int q = 0; q < ng; ++q) s += (transpose ? op[q * kMaxNg + c] : op[c * kMaxNg + q]) * src[base + q * stride];
    dst[p] = accumulate ? dst[p] + s : s;
  }
  __syncwarp();
}

// Child-to-parent: M^P = sum_C (T^{a_x} (x) T^{a_y} (x) T^{a_z}) M^C, one parent per warp,
// for every expanded box (an internal cell, or a leaf or virtual box whose
// children are needed as sources): its children hold all its particles, so by
// the moment-matching identity of Sec. 2.3 this equals its P2G to rounding.
__global__ void __launch_bounds__(kGThreads) k_m2m(int64_t b, int64_t e, GridletTables tb,
                                                  const uint8_t *__restrict__ flags,
                                                  const int *__restrict__ child, int64_t off2,
                                                  float *__restrict__ grid, const uint64_t *__restrict__ key,
                                                  int level, int *__restrict__ amax, int nlev) {
  __shared__ float T[2][kMaxNg * kMaxNg];
  __shared__ float bufA[kGWarps][512], bufB[kGWarps][512], res[kGWarps][512];
  for (int i = threadIdx.x; i < 2 * kMaxNg * kMaxNg; i += blockDim.x)
    T[i / (kMaxNg * kMaxNg)][i % (kMaxNg * kMaxNg)] = tb.t1[i / (kMaxNg * kMaxNg)][(i / kMaxNg) % kMaxNg][i % kMaxNg];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t box = b + (int64_t)blockIdx.x * kGWarps + w;
  if (box >= e || !(flags[box] & kExpand)) return;
  const int ng = tb.ng, m3 = ng * ng * ng;
  for (int p = lane; p < m3; p += 32) res[w][p] = 0.f;
  for (int o = 0; o < 8; ++o) {
    const int c = child[box * 8 + o];
    if (c < 0) continue;
    const float *src = grid + (int64_t)(c - off2) * m3;
    for (int p = lane; p < m3; p += 32) bufA[w][p] = src[p];
    __syncwarp();
    apply_axis(T[o & 1], false, 0, ng, bufA[w], bufB[w], false);
    apply_axis(T[(o >> 1) & 1], false, 1, ng, bufB[w], bufA[w], false);
    apply_axis(T[(o >> 2) & 1], false, 2, ng, bufA[w], res[w], true);
  }
  float *dst = grid + (int64_t)(box - off2) * m3;
  float a = 0.f;
  for (int p = lane; p < m3; p += 32) {
    dst[p] = res[w][p];
    a = fmaxf(a, fabsf(res[w][p]));
  }
  row_amax(amax, a, key, box, level, nlev);
}

// Ng = 4 child-to-parent, one parent per warp, with the transform factored
// over the child octants: M^P = sum_cz Tz (sum_cy Ty (sum_cx Tx M^(cx,cy,cz)))
// (T^{a} of the x, y, z axes as in k_m2m). The 8 children are loaded at once;
// the x stage forms 4 gridlets (summed over cx), y forms 2, z the parent.
// kW warps (gridlets) per CTA: a launch shape the tuner picks (2, 4 or 8);
// each warp's arithmetic is the same whatever kW.
template <int kW>
__global__ void __launch_bounds__(kW * 32) k_m2m4(int64_t b, int64_t e, GridletTables tb,
                                                         const uint8_t *__restrict__ flags,
                                                         const int *__restrict__ child, int64_t off2,
                                                         float *__restrict__ grid, const uint64_t *__restrict__ key,
                                                         int level, int *__restrict__ amax, int nlev) {
  __shared__ float T[2][4][4];
  __shared__ float ch[kW][8][64], X[kW][4][64], Y[kW][2][64];
  if (threadIdx.x < 32) T[threadIdx.x >> 4][(threadIdx.x >> 2) & 3][threadIdx.x & 3] =
      tb.t1[threadIdx.x >> 4][(threadIdx.x >> 2) & 3][threadIdx.x & 3];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t box = b + (int64_t)blockIdx.x * kW + w;
  if (box >= e || !(flags[box] & kExpand)) return;
  {
    // child o = lane / 4, 16 values each
    const int o = lane >> 2, sub = lane & 3;
    const int c = child[box * 8 + o];
    float4 v[4];
    if (c >= 0) {
      const float4 *src = reinterpret_cast<const float4 *>(grid + (int64_t)(c - off2) * 64 + 16 * sub);
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = src[k];
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float4 *dst = reinterpret_cast<float4 *>(&ch[w][o][16 * sub]);
#pragma unroll
    for (int k = 0; k < 4; ++k) dst[k] = v[k];
  }
  __syncwarp();
  // x: X[cy + 2 cz][p] = sum_cx sum_qx T[cx][px][qx] ch[cx + 2cy + 4cz][qx, py, pz]
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int idx = r * 32 + lane, g = idx >> 6, p = idx & 63, px = p & 3, rowb = p - px;
    float acc = 0.f;
#pragma unroll
    for (int cx = 0; cx < 2; ++cx)
#pragma unroll
      for (int qx = 0; qx < 4; ++qx) acc = fmaf(T[cx][px][qx], ch[w][cx + 2 * g][rowb + qx], acc);
    X[w][g][p] = acc;
  }
  __syncwarp();
  // y: Y[cz][p] = sum_cy sum_qy T[cy][py][qy] X[cy + 2cz][px, qy, pz]
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int idx = r * 32 + lane, cz = idx >> 6, p = idx & 63, py = (p >> 2) & 3, base = p - 4 * py;
    float acc = 0.f;
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int qy = 0; qy < 4; ++qy) acc = fmaf(T[cy][py][qy], X[w][cy + 2 * cz][base + 4 * qy], acc);
    Y[w][cz][p] = acc;
  }
  __syncwarp();
  // z: M^P[p] = sum_cz sum_qz T[cz][pz][qz] Y[cz][px, py, qz]
  float *out = grid + (int64_t)(box - off2) * 64;
  float a = 0.f;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int p = r * 32 + lane, pz = p >> 4, base = p & 15;
    float acc = 0.f;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int qz = 0; qz < 4; ++qz) acc = fmaf(T[cz][pz][qz], Y[w][cz][base + 16 * qz], acc);
    out[p] = acc;
    a = fmaxf(a, fabsf(acc));
  }
  row_amax(amax, a, key, box, level, nlev);
}

// Ng = 4 parent-to-child (Sec. 2.4), one target per warp with the three axis
// passes unrolled in FP32: loc_C = (Tx^T (x) Ty^T (x) Tz^T) loc_P + own
// values, kept as (constant, deviations) as in k_l2l_df.
template <int kW>
__global__ void __launch_bounds__(kW * 32) k_l2l4(int64_t tb0, int64_t tb1, int level, GridletTables tab,
                                                         const int *__restrict__ tgt_box,
                                                         const int *__restrict__ box_tgt,
                                                         const int *__restrict__ parent,
                                                         const uint64_t *__restrict__ key,
                                                         const float *__restrict__ raw, float *__restrict__ loc,
                                                         float *__restrict__ locc, const float *__restrict__ m2lc) {
  __shared__ float T[2][4][4];
  __shared__ float A[kW][64], B[kW][64];
  if (threadIdx.x < 32) T[threadIdx.x >> 4][(threadIdx.x >> 2) & 3][threadIdx.x & 3] =
      tab.t1[threadIdx.x >> 4][(threadIdx.x >> 2) & 3][threadIdx.x & 3];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t t = tb0 + (int64_t)blockIdx.x * kW + w;
  if (t >= tb1) return;
  const float2 own = reinterpret_cast<const float2 *>(raw + t * 64)[lane];
  float r0 = own.x, r1 = own.y;  // nodes 2 lane, 2 lane + 1
  float cpar = 0.f;
  if (level >= 3) {
    const int box = tgt_box[t];
    const int tp = box_tgt[parent[box]];
    const int o = (int)(key[box] & 7u);
    const int ax = o & 1, ay = (o >> 1) & 1, az = (o >> 2) & 1;
    const float2 pv = reinterpret_cast<const float2 *>(loc + (int64_t)tp * 64)[lane];
    cpar = locc[tp];
    A[w][2 * lane] = pv.x;
    A[w][2 * lane + 1] = pv.y;
    __syncwarp();
    // x: B[p] = sum_q T[ax][q][px] A[q, py, pz]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int p = 2 * lane + k, px = p & 3, rowb = p - px;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(T[ax][q][px], A[w][rowb + q], acc);
      B[w][p] = acc;
    }
    __syncwarp();
    // y: A[p] = sum_q T[ay][q][py] B[px, q, pz]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int p = 2 * lane + k, py = (p >> 2) & 3, base = p - 4 * py;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(T[ay][q][py], B[w][base + 4 * q], acc);
      A[w][p] = acc;
    }
    __syncwarp();
    // z: own += sum_q T[az][q][pz] A[px, py, q]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int p = 2 * lane + k, pz = p >> 4, base = p & 15;
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) acc = fmaf(T[az][q][pz], A[w][base + 16 * q], acc);
      if (k == 0) r0 += acc; else r1 += acc;
    }
  }
  float s = r0 + r1;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  const float mean = s / 64.f;
  reinterpret_cast<float2 *>(loc + t * 64)[lane] = make_float2(r0 - mean, r1 - mean);
  if (lane == 0) locc[t] = cpar + (mean + m2lc[t]);
}

// Double-float arithmetic (a value is hi + lo, |lo| <= ulp(hi) / 2) on the
// FP32 pipe, for the parent-to-child pass of the orders other than 4: at
// Ng >= 5 the interpolation from the parent's nodes to the child's amplifies
// the FP32 rounding of plain products into the force beyond 1e-5, while FP64
// arithmetic runs about 70 times slower than FP32 on this GPU.
struct dfloat {
  float h, l;
};
__device__ __forceinline__ dfloat df_quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const float s = a.h + b.h, bb = s - a.h;
  const float e = (a.h - (s - bb)) + (b.h - bb);  // two-sum error of a.h + b.h
  return df_quick_two_sum(s, e + (a.l + b.l));
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);  // exact error of the product
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return df_quick_two_sum(p, e);
}

// One axis pass in double-float: dst[.., p_axis, ..] = sum_q T[q][p] src[.., q, ..]
// (the transposed 1-D operator, parent-to-child), T = hi + lo.
__device__ __forceinline__ void apply_axis_df(const float *__restrict__ th, const float *__restrict__ tl, int axis,
                                              int ng, const dfloat *src, dfloat *dst) {
  const int lane = threadIdx.x & 31, m3 = ng * ng * ng;
  const int stride = axis == 0 ? 1 : (axis == 1 ? ng : ng * ng);
  for (int p = lane; p < m3; p += 32) {
    const int c = (p / stride) % ng;
    const int base = p - c * stride;
    dfloat s = {0.f, 0.f};
    for (int q = 0; q < ng; ++q)
      s = df_add(s, df_mul({th[q * kMaxNg + c], tl[q * kMaxNg + c]}, src[base + q * stride]));
    dst[p] = s;
  }
  __syncwarp();
}

// Parent-to-child plus the target's own source-to-target values (Sec. 2.4),
// for the orders other than 4, one target per warp. The local is kept as
// (constant, deviations): the interpolation reproduces constants exactly (the
// Lagrange weights sum to one), so the constant is carried separately and the
// FP32 deviations only hold the variation across the cell. The interpolation,
// the addition of the target's own values and the mean are evaluated in
// double-float.
constexpr int kDfWarps = 2;
__global__ void __launch_bounds__(32 * kDfWarps) k_l2l_df(int64_t tb0, int64_t tb1, int level, GridletTables tab,
                                                       const int *__restrict__ tgt_box,
                                                       const int *__restrict__ box_tgt,
                                                       const int *__restrict__ parent,
                                                       const uint64_t *__restrict__ key,
                                                       const float *__restrict__ raw, float *__restrict__ loc,
                                                       float *__restrict__ locc, const float *__restrict__ m2lc) {
  __shared__ float Th[2][kMaxNg * kMaxNg], Tl[2][kMaxNg * kMaxNg];
  __shared__ dfloat bufA[kDfWarps][512], bufB[kDfWarps][512];
  for (int i = threadIdx.x; i < 2 * kMaxNg * kMaxNg; i += blockDim.x) {
    const int sgn = i / (kMaxNg * kMaxNg), pq = i % (kMaxNg * kMaxNg);
    Th[sgn][pq] = tab.t1[sgn][pq / kMaxNg][pq % kMaxNg];
    Tl[sgn][pq] = tab.t1lo[sgn][pq / kMaxNg][pq % kMaxNg];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t t = tb0 + (int64_t)blockIdx.x * kDfWarps + w;
  if (t >= tb1) return;
  const int ng = tab.ng, m3 = ng * ng * ng;
  dfloat *res = bufB[w];
  float cpar = 0.f;
  if (level >= 3) {
    const int box = tgt_box[t];
    const int tp = box_tgt[parent[box]];
    const int o = (int)(key[box] & 7u);
    const float *pl = loc + (int64_t)tp * m3;
    for (int p = lane; p < m3; p += 32) bufA[w][p] = {pl[p], 0.f};
    __syncwarp();
    apply_axis_df(Th[o & 1], Tl[o & 1], 0, ng, bufA[w], bufB[w]);
    apply_axis_df(Th[(o >> 1) & 1], Tl[(o >> 1) & 1], 1, ng, bufB[w], bufA[w]);
    apply_axis_df(Th[(o >> 2) & 1], Tl[(o >> 2) & 1], 2, ng, bufA[w], bufB[w]);
    for (int p = lane; p < m3; p += 32) res[p] = df_add(res[p], {raw[t * m3 + p], 0.f});
    cpar = locc[tp];
  } else {
    for (int p = lane; p < m3; p += 32) res[p] = {raw[t * m3 + p], 0.f};
  }
  __syncwarp();
  dfloat s = {0.f, 0.f};
  for (int p = lane; p < m3; p += 32) s = df_add(s, res[p]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
    s = df_add(s, {__shfl_xor_sync(0xffffffffu, s.h, off), __shfl_xor_sync(0xffffffffu, s.l, off)});
  // mean = s / m3 in double-float: quotient, then the remainder's correction
  const float qh = s.h / (float)m3;
  const float rem = fmaf(-qh, (float)m3, s.h) + s.l;
  const dfloat mean = df_quick_two_sum(qh, rem / (float)m3);
  float *mine = loc + t * m3;
  for (int p = lane; p < m3; p += 32) {
    const dfloat d = df_add(res[p], {-mean.h, -mean.l});
    mine[p] = d.h + d.l;
  }
  if (lane == 0) locc[t] = cpar + (mean.h + m2lc[t]);
}

// 1-D Lagrange weights and derivatives, FP32 (NG as for lagrange_d).
template <int NG>
__device__ __forceinline__ void lagrange_f(const GridletTables &tb, float t, float *w, float *dw) {
  const int ng = NG > 0 ? NG : tb.ng;
  float diff[kMaxNg];
#pragma unroll
  for (int k = 0; k < (NG > 0 ? NG : kMaxNg); ++k)
    if (k < ng) diff[k] = t - tb.node[k];
#pragma unroll
  for (int j = 0; j < (NG > 0 ? NG : kMaxNg); ++j) {
    if (j >= ng) break;
    float v = tb.inv_den[j], d = 0.f;
#pragma unroll
    for (int k = 0; k < (NG > 0 ? NG : kMaxNg); ++k) {
      if (k >= ng) break;
      if (k == j) continue;
      d = d * diff[k] + v;
      v *= diff[k];
    }
    w[j] = v;
    dw[j] = d;
  }
}

// Far field at every particle from its leaf's local gridlet (one thread per
// sorted particle, FP32 throughout): phi = c + sum_p delta_p prod ell,
// a = -(2^l / S) sum_p delta_p grad_xi prod ell (Eq. phix and its gradient).
template <int NG>
__global__ void __launch_bounds__(kThreads, NG == 4 ? 6 : 1) k_g2p(int64_t n, const int *__restrict__ pbox,
                                                  const int *__restrict__ box_tgt, LevelTable lt,
                                                  GridletTables tb, float inv_side,
                                                  const uint64_t *__restrict__ key,
                                                  const float4 *__restrict__ uhi, const float4 *__restrict__ ulo,
                                                  const float *__restrict__ loc,
                                                  const float *__restrict__ locc,
                                                  float4 *__restrict__ far) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int box = pbox[i];
  const int t = box_tgt[box];
  if (t < 0) {  // a leaf above level 2 has no far field
    far[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const int ng = NG > 0 ? NG : tb.ng;
  const int l = level_of(lt, box);
  const uint64_t k = key[box] & ((1ull << (3 * l)) - 1ull);
  const float sc = (float)(1u << l);
  const float4 h = uhi[i], q = ulo[i];
  float wv[3][kMaxNg], dw[3][kMaxNg];
  lagrange_f<NG>(tb, cell_coord(h.x, q.x, sc, (float)compact3(k) + 0.5f), wv[0], dw[0]);
  lagrange_f<NG>(tb, cell_coord(h.y, q.y, sc, (float)compact3(k >> 1) + 0.5f), wv[1], dw[1]);
  lagrange_f<NG>(tb, cell_coord(h.z, q.z, sc, (float)compact3(k >> 2) + 0.5f), wv[2], dw[2]);
  const float *dl = loc + (int64_t)t * ng * ng * ng;
  // contracted axis by axis: x for every (y, z) row (the value and its x
  // derivative), then y for every z (value, y and x derivatives), then z
  float f = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
  for (int pz = 0; pz < (NG > 0 ? NG : kMaxNg); ++pz) {
    if (pz >= ng) break;
    float fy = 0.f, yy = 0.f, xy = 0.f;
#pragma unroll
    for (int py = 0; py < (NG > 0 ? NG : kMaxNg); ++py) {
      if (py >= ng) break;
      const float *row = dl + ng * (py + ng * pz);
      float fx = 0.f, xx = 0.f;
      if constexpr (NG == 4) {
        // a row is one 16-byte load (four lanes of a warp on different leaves
        // cost one L1 wavefront per load instead of four)
        const float4 v = __ldg(reinterpret_cast<const float4 *>(row));
        fx = fmaf(v.w, wv[0][3], fmaf(v.z, wv[0][2], fmaf(v.y, wv[0][1], v.x * wv[0][0])));
        xx = fmaf(v.w, dw[0][3], fmaf(v.z, dw[0][2], fmaf(v.y, dw[0][1], v.x * dw[0][0])));
      } else {
#pragma unroll
        for (int px = 0; px < (NG > 0 ? NG : kMaxNg); ++px) {
          if (px >= ng) break;
          const float v = __ldg(row + px);
          fx = fmaf(v, wv[0][px], fx);
          xx = fmaf(v, dw[0][px], xx);
        }
      }
      fy = fmaf(fx, wv[1][py], fy);
      yy = fmaf(fx, dw[1][py], yy);
      xy = fmaf(xx, wv[1][py], xy);
    }
    f = fmaf(fy, wv[2][pz], f);
    gz = fmaf(fy, dw[2][pz], gz);
    gy = fmaf(yy, wv[2][pz], gy);
    gx = fmaf(xy, wv[2][pz], gx);
  }
  const float invL = sc * inv_side;
  far[i] = make_float4(__ldg(locc + t) + f, -gx * invL, -gy * invL, -gz * invL);
}

// Far field for the orders other than 4, as k_g2p but with the weights and
// the gradient's contraction in double-float: at Ng >= 5 the derivatives of
// the Lagrange basis are large and of both signs, so plain FP32 products and
// sums lose the deviations' precision (FP64 runs about 70 times slower than
// FP32 on this GPU). The cell coordinate xi = (h 2^l - c) + lo 2^l is exact as
// two floats; the weights follow the product form ell_j = prod_{k != j}
// (xi - x_k) / (x_j - x_k) and its product-rule derivative; the contraction is
// factorised x, then y, then z. The potential keeps the FP32 contraction.
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfloat df_mul_f(dfloat a, float b) {
  const float p = a.h * b;
  return df_quick_two_sum(p, fmaf(a.h, b, -p) + a.l * b);
}
template <int NG>
__device__ __forceinline__ void lagrange_df(const GridletTables &tb, dfloat xi, float *w, dfloat *wd,
                                            dfloat *dd) {
  const int ng = NG > 0 ? NG : tb.ng;
  dfloat diff[kMaxNg];
#pragma unroll
  for (int k = 0; k < (NG > 0 ? NG : kMaxNg); ++k)
    if (k < ng) diff[k] = df_add(xi, {-tb.node[k], -tb.node_lo[k]});
#pragma unroll
  for (int j = 0; j < (NG > 0 ? NG : kMaxNg); ++j) {
    if (j >= ng) break;
    dfloat v = {tb.inv_den[j], tb.inv_den_lo[j]}, d = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < (NG > 0 ? NG : kMaxNg); ++k) {
      if (k >= ng) break;
      if (k == j) continue;
      d = df_add(df_mul(d, diff[k]), v);
      v = df_mul(v, diff[k]);
    }
    w[j] = v.h + v.l;
    wd[j] = v;
    dd[j] = d;
  }
}

template <int NG>
__global__ void __launch_bounds__(kThreads) k_g2p_df(int64_t n, const int *__restrict__ pbox,
                                                     const int *__restrict__ box_tgt, LevelTable lt,
                                                     GridletTables tb, float inv_side,
                                                     const uint64_t *__restrict__ key,
                                                     const float4 *__restrict__ uhi, const float4 *__restrict__ ulo,
                                                     const float *__restrict__ loc,
                                                     const float *__restrict__ locc, float4 *__restrict__ far) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int box = pbox[i];
  const int t = box_tgt[box];
  if (t < 0) {  // a leaf above level 2 has no far field
    far[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  constexpr int kN = NG > 0 ? NG : kMaxNg;
  const int ng = NG > 0 ? NG : tb.ng;
  const int l = level_of(lt, box);
  const uint64_t k = key[box] & ((1ull << (3 * l)) - 1ull);
  const float sc = (float)(1u << l);
  const float4 h = uhi[i], q = ulo[i];
  float w[3][kN];
  dfloat wd[3][kN], dd[3][kN];
  lagrange_df<NG>(tb, df_two_sum(fmaf(h.x, sc, -((float)compact3(k) + 0.5f)), q.x * sc), w[0], wd[0], dd[0]);
  lagrange_df<NG>(tb, df_two_sum(fmaf(h.y, sc, -((float)compact3(k >> 1) + 0.5f)), q.y * sc), w[1], wd[1], dd[1]);
  lagrange_df<NG>(tb, df_two_sum(fmaf(h.z, sc, -((float)compact3(k >> 2) + 0.5f)), q.z * sc), w[2], wd[2], dd[2]);
  const float *dl = loc + (int64_t)t * ng * ng * ng;
  float f = 0.f;
  dfloat gx = {0.f, 0.f}, gy = {0.f, 0.f}, gz = {0.f, 0.f};
#pragma unroll
  for (int pz = 0; pz < kN; ++pz) {
    if (pz >= ng) break;
    dfloat zx = {0.f, 0.f}, zy = {0.f, 0.f}, z0 = {0.f, 0.f};  // sums over y of the x-sums
#pragma unroll
    for (int py = 0; py < kN; ++py) {
      if (py >= ng) break;
      const float *row = dl + ng * (py + ng * pz);
      dfloat r0 = {0.f, 0.f}, r1 = {0.f, 0.f};  // sum_x v w_x, sum_x v w_x'
      float f0 = 0.f;
#pragma unroll
      for (int px = 0; px < kN; ++px) {
        if (px >= ng) break;
        const float v = __ldg(row + px);
        f0 = fmaf(v, w[0][px], f0);
        r0 = df_add(r0, df_mul_f(wd[0][px], v));
        r1 = df_add(r1, df_mul_f(dd[0][px], v));
      }
      f = fmaf(f0, w[1][py] * w[2][pz], f);
      zx = df_add(zx, df_mul(r1, wd[1][py]));
      zy = df_add(zy, df_mul(r0, dd[1][py]));
      z0 = df_add(z0, df_mul(r0, wd[1][py]));
    }
    gx = df_add(gx, df_mul(zx, wd[2][pz]));
    gy = df_add(gy, df_mul(zy, wd[2][pz]));
    gz = df_add(gz, df_mul(z0, dd[2][pz]));
  }
  const float invL = sc * inv_side;
  far[i] = make_float4(__ldg(locc + t) + f, -(gx.h + gx.l) * invL, -(gy.h + gy.l) * invL, -(gz.h + gz.l) * invL);
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float x) {
  const float y = x - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// A particle's position relative to the target leaf's centre as a rounded
// FP32 value r and its exact residual e (the hi part relative to the centre
// plus the lo residual of the unit-cube coordinate, r + e = the sum).
__device__ __forceinline__ float2 rel_split(float h, float c0, float lo) {
  const float hr = h - c0;
  const float r = hr + lo;
  return make_float2(r, (hr - r) + lo);
}

// Near-field kernel forms: 0 Plummer (Newton with eps = 0), 1 Yukawa, 2 a
// user kernel from its table (green.cu). Pairs are summed in unit-cube
// coordinates; the closed forms are scaled back by 1/S (potential) and 1/S^2
// (acceleration) once per target, the table holds physical g and the force
// factor -g'(r) / r_u directly.
struct NearKernel {
  float eps2;         // (eps / S)^2, forms 0 and 1
  float inv_lambda;   // S / lambda, form 1
  const float4 *tab;  // form 2: per segment the cubic coefficients of g, then of the force factor
};

// 1 / sqrt(x) by the hardware approximation (rsqrt.approx, relative error
// below 2^-22.9) with subnormal inputs flushed to zero: a squared pair
// distance below 2^-126 of the domain side squared counts as 0 (the pair
// coincides), which spares the subnormal rescaling of every pair.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// m g(r) and m F(r), F the force factor (a_i += m F (x_j - x_i)), of a pair at
// squared distance r2 (softening included for forms 0 and 1).
template <int KIND>
__device__ __forceinline__ void pair_coef(const NearKernel &nk, float r2, float m, float &mg, float &mf) {
  if constexpr (KIND == 0) {
    const float ir = rsqrt_ftz(r2);
    mg = m * ir;
    mf = mg * ir * ir;
  } else if constexpr (KIND == 1) {
    const float ir = rsqrt_ftz(r2);
    const float sl = r2 * ir * nk.inv_lambda;  // s / lambda
    mg = m * ir * __expf(-sl);
    mf = mg * ir * ir * (1.f + sl);
  } else {
    // segment: (exponent - E0) * 32 + the top 5 mantissa bits of r2; the
    // position in it: the remaining 18 mantissa bits
    const unsigned b = __float_as_uint(r2);
    int seg = (int)(b >> 18) - ((127 + kNearTabE0) << 5);
    float t = (float)(b & 0x3FFFFu) * (1.f / 262144.f);
    if (seg < 0) {
      seg = 0;
      t = 0.f;
    } else if (seg >= kNearTabOctaves * kNearTabSeg) {
      seg = kNearTabOctaves * kNearTabSeg - 1;
      t = 1.f;
    }
    const float4 cg = __ldg(nk.tab + 2 * seg), cf = __ldg(nk.tab + 2 * seg + 1);
    mg = m * fmaf(fmaf(fmaf(cg.w, t, cg.z), t, cg.y), t, cg.x);
    mf = m * fmaf(fmaf(fmaf(cf.w, t, cf.z), t, cf.y), t, cf.x);
  }
}

// One source's contribution to a target, accumulated into a short plain-FP32
// block sum. pair_fast takes the difference of the rounded relative positions
// (error below 2^-23 of the leaf side) and returns r^2 for the block's check;
// pair_exact takes (r_s - r_t) + (e_s - e_t), which keeps FP32 precision
// relative to the pair distance however small it is, and skips the target
// itself. sr.w holds the mass, se.w the particle index.
template <int KIND>
__device__ __forceinline__ float pair_fast(const float4 &tr, const float4 &s, const NearKernel &nk, float &bp,
                                           float &bx, float &by, float &bz) {
  const float dx = s.x - tr.x, dy = s.y - tr.y, dz = s.z - tr.z;
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, nk.eps2)));
  float mg, mf;
  pair_coef<KIND>(nk, r2, s.w, mg, mf);
  bp -= mg;
  bx = fmaf(mf, dx, bx);
  by = fmaf(mf, dy, by);
  bz = fmaf(mf, dz, bz);
  return r2;
}

template <int KIND>
__device__ __forceinline__ void pair_exact(const float4 &tr, const float4 &te, const float4 &s, const float4 &e,
                                           const NearKernel &nk, float &bp, float &bx, float &by, float &bz) {
  const float dx = (s.x - tr.x) + (e.x - te.x), dy = (s.y - tr.y) + (e.y - te.y), dz = (s.z - tr.z) + (e.z - te.z);
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, nk.eps2)));
  float mg, mf;
  if constexpr (KIND == 0) {
    float ir = rsqrt_ftz(r2);
    if (__float_as_int(e.w) == __float_as_int(te.w)) ir = 0.f;  // the target itself
    mg = s.w * ir;
    mf = mg * ir * ir;
  } else {
    pair_coef<KIND>(nk, r2, s.w, mg, mf);
    if (__float_as_int(e.w) == __float_as_int(te.w)) mg = mf = 0.f;  // the target itself
  }
  bp -= mg;
  bx = fmaf(mf, dx, bx);
  by = fmaf(mf, dy, by);
  bz = fmaf(mf, dz, bz);
}

// Near zone by direct summation (Sec. 1, item 1), one warp per work item: an
// item is a leaf's targets against a contiguous part of the concatenation of
// its near boxes' particles. The item's sources are staged in shared memory in
// chunks (rounded position relative to the target leaf's centre and mass,
// exact residual and index; each source's range found from a bit mask of the
// range starts in its 32-source window), so the pair loop is one flat loop; floor(32 / nt) lanes share a target and split
// the chunk; blocks of eight pairs are summed in plain FP32 and the block sums
// are Kahan compensated. A leaf with one item, and an item of a leaf split by
// targets (32 of them against all near sources), writes far + near to the
// caller's order; a leaf split over sources writes partial sums for
// k_p2p_combine. Warps take items from a counter (zeroed before the launch) and
// the grid holds as many blocks as are resident at once, so a warp whose item
// ends early starts the next one instead of idling until its block retires.
constexpr int kP2PChunk = 128;
// Targets of an item's first pass, by its number of targets (the rest, if
// any, in a second pass): the split that minimises the passes' time per source,
// 1 / lanes per target of each pass plus its staging (about 0.09 of a one-lane
// pass), over the two-pass splits and the single pass
__constant__ unsigned char c_p2p_first_pass[33] = {0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 3,  4,  13, 14, 15, 16,
                                                   1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 27, 28, 29, 30, 31, 32};

template <int KIND>
__global__ void __launch_bounds__(kThreads, 4) k_p2p(int64_t nitem, const int *__restrict__ item_leaf,
                                                  const int *__restrict__ item_s0, const int *__restrict__ item_s1,
                                                  const int *__restrict__ item_t,
                                                  const int *__restrict__ leaf_nitem,
                                                  const int *__restrict__ leaf_item0,
                                                  const int *__restrict__ leaf_part0,
                                                  const int *__restrict__ leaf_box, const int *__restrict__ nb,
                                                  const int *__restrict__ beg, const int *__restrict__ end,
                                                  const float4 *__restrict__ hi, const float4 *__restrict__ lo,
                                                  const float4 *__restrict__ far,
                                                  const uint32_t *__restrict__ perm, const uint64_t *__restrict__ key,
                                                  LevelTable lt, NearKernel nk, float sc_phi,
                                                  float sc_acc, float *__restrict__ out_phi, float *__restrict__ out_acc,
                                                  float4 *__restrict__ part, unsigned long long *__restrict__ next) {
  __shared__ float4 red[kWarpsPerBlock][32];
  __shared__ int2 rng[kWarpsPerBlock][27];
  __shared__ float4 srh[kWarpsPerBlock][kP2PChunk], srl[kWarpsPerBlock][kP2PChunk];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (;;) {
  unsigned long long it0 = 0;
  if (lane == 0) it0 = atomicAdd(next, 1ull);
  const int64_t it = (int64_t)__shfl_sync(0xffffffffu, it0, 0);
  if (it >= nitem) return;
  __syncwarp();
  const int leaf = item_leaf[it];
  const int box = leaf_box[leaf];
  // the item's near boxes with particles, compacted: rng[w][k], k < nr, is
  // the k-th one's first particle and the index of that particle in the
  // concatenation of their particle ranges (strictly increasing in k)
  int nr, own0;
  {
    int b = 0, c = 0;
    if (lane < 27) {
      const int q = nb[(int64_t)box * 27 + lane];
      if (q >= 0) {
        b = beg[q];
        c = end[q] - b;
      }
    }
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    // the target leaf's own particles start at this concatenated index (its
    // own box is neighbour 13)
    own0 = __shfl_sync(0xffffffffu, inc - c, 13);
    const unsigned ne = __ballot_sync(0xffffffffu, c > 0);
    nr = __popc(ne);
    if (c > 0) rng[w][__popc(ne & ((1u << lane) - 1u))] = make_int2(b, inc - c);
    __syncwarp();
  }
  const int s0 = item_s0[it], s1 = item_s1[it];
  const int tb = beg[box], te = end[box], nt = te - tb;
  // this item's targets: the whole leaf, or 32 of a leaf split by targets
  const int tsel = item_t[it];
  const int ta = tsel < 0 ? tb : tb + tsel, tz = tsel < 0 ? te : min(te, tb + tsel + 32), nti = tz - ta;
  // the target leaf's centre in unit-cube coordinates (exact in FP32)
  float cx0, cy0, cz0;
  {
    const int l = level_of(lt, box);
    const uint64_t kk = key[box] & ((1ull << (3 * l)) - 1ull);
    const float inv = 1.f / (float)(1u << l);
    cx0 = ((float)compact3(kk) + 0.5f) * inv;
    cy0 = ((float)compact3(kk >> 1) + 0.5f) * inv;
    cz0 = ((float)compact3(kk >> 2) + 0.5f) * inv;
  }
  const int nitems = leaf_nitem[leaf];
  float near2;
  {
    const float side = 1.f / (float)(1u << level_of(lt, box));  // the leaf's side (unit cube)
    near2 = nk.eps2 + side * side * (1.f / 64.f);  // r^2 of a pair 1/8 of the side apart
  }
  const int kidx = (int)(it - leaf_item0[leaf]);
  // one or two passes over the targets, each with floor(32 / its targets)
  // lanes per target (at most 16): a leaf of 17 targets takes 1 then 16 (16
  // then 2 lanes per target) instead of 17 at 1 lane
  const int split = nti <= 32 ? c_p2p_first_pass[nti] : 32;
  for (int pass = 0; pass < 2; ++pass) {
  const int pa = pass == 0 ? ta : ta + split, pz = pass == 0 ? ta + split : tz;
  if (pa >= pz) break;
  const int G = pz - pa >= 32 ? 1 : min(16, 32 / (pz - pa));
  const int per = 32 / G;
  for (int t0 = pa; t0 < pz; t0 += per) {
    const int slot = lane / G, sub = lane % G;
    const int ti = t0 + slot;
    const bool active = slot < per && ti < pz;
    float4 th = make_float4(0.f, 0.f, 0.f, 0.f), tl = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));
    if (active) {
      const float4 h = hi[ti], q = lo[ti];
      const float2 x = rel_split(h.x, cx0, q.x), y = rel_split(h.y, cy0, q.y), z = rel_split(h.z, cz0, q.z);
      th = make_float4(x.x, y.x, z.x, 0.f);
      tl = make_float4(x.y, y.y, z.y, __int_as_float(ti));
    }
    float sp = 0.f, cp = 0.f, sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
    for (int c0 = s0; c0 < s1; c0 += kP2PChunk) {
      const int cn = min(kP2PChunk, s1 - c0);
      __syncwarp();
      for (int k0 = 0; k0 < cn; k0 += 64) {
        int j[2];
        float4 h[2], o[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          // the range of concatenated index q = s + lane: the ranges that start
          // before the window s ... s + 31, plus those starting in it up to q
          const int s = c0 + k0 + 32 * u, q = s + lane;
          const int ck = lane < nr ? rng[w][lane].y : 0x7fffffff;
          const int before = __popc(__ballot_sync(0xffffffffu, ck < s));
          const int d = ck - s;
          const unsigned mask = __reduce_or_sync(0xffffffffu, d >= 0 && d < 32 ? 1u << d : 0u);
          const int r = before - 1 + __popc(mask & (0xffffffffu >> (31 - lane)));
          const int2 v = rng[w][r];
          j[u] = q < c0 + cn ? v.x + (q - v.y) : v.x;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          h[u] = hi[j[u]];
          o[u] = lo[j[u]];
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = k0 + lane + 32 * u;
          if (k < cn) {
            const float2 x = rel_split(h[u].x, cx0, o[u].x), y = rel_split(h[u].y, cy0, o[u].y),
                         z = rel_split(h[u].z, cz0, o[u].z);
            srh[w][k] = make_float4(x.x, y.x, z.x, h[u].w);
            srl[w][k] = make_float4(x.y, y.y, z.y, __int_as_float(j[u]));
          }
        }
      }
      __syncwarp();
      if (active) {
        // the chunk positions of this pass's targets as sources: a block that
        // reaches them holds some lane's own particle and is summed exactly
        // at once
        const int self0 = own0 + (t0 - tb) - c0, self1 = own0 + (min(t0 + per, pz) - tb) - c0;
        int k = sub;
        for (; k + 7 * G < cn; k += 8 * G) {
          // eight pairs from the rounded positions; if some lane of the warp
          // has a pair closer than near2 in them the block is summed again
          // exactly
          float bp = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
          const int kb = k - sub;  // the warp's block: positions kb ... kb + 8 G - 1
          bool exact = kb < self1 && kb + 8 * G > self0;
          if (!exact) {
            float r2min = 3.4e38f;
#pragma unroll
            for (int u = 0; u < 8; ++u) r2min = fminf(r2min, pair_fast<KIND>(th, srh[w][k + u * G], nk, bp, bx, by, bz));
            exact = __any_sync(__activemask(), r2min <= near2);
          }
          if (exact) {
            bp = bx = by = bz = 0.f;
#pragma unroll 4
            for (int u = 0; u < 8; ++u) {
              const int kk = k + u * G;
              pair_exact<KIND>(th, tl, srh[w][kk], srl[w][kk], nk, bp, bx, by, bz);
            }
          }
          kahan_add(sp, cp, bp);
          kahan_add(sx, cx, bx);
          kahan_add(sy, cy, by);
          kahan_add(sz, cz, bz);
        }
        float bp = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
        for (; k < cn; k += G) pair_exact<KIND>(th, tl, srh[w][k], srl[w][k], nk, bp, bx, by, bz);
        kahan_add(sp, cp, bp);
        kahan_add(sx, cx, bx);
        kahan_add(sy, cy, by);
        kahan_add(sz, cz, bz);
      }
    }
    red[w][lane] = make_float4(sp - cp, sx - cx, sy - cy, sz - cz);
    __syncwarp();
    if (active && sub == 0) {
      float4 v = red[w][lane];
      for (int g = 1; g < G; ++g) {
        const float4 o = red[w][lane + g];
        v.x += o.x;
        v.y += o.y;
        v.z += o.z;
        v.w += o.w;
      }
      if (nitems == 1 || tsel >= 0) {  // all of this target's near sources
        const float4 f = far[ti];
        const uint32_t o = perm[ti];
        if (out_phi) out_phi[o] = fmaf(v.x, sc_phi, f.x);
        if (out_acc) {
          out_acc[3 * (int64_t)o] = fmaf(v.y, sc_acc, f.y);
          out_acc[3 * (int64_t)o + 1] = fmaf(v.z, sc_acc, f.z);
          out_acc[3 * (int64_t)o + 2] = fmaf(v.w, sc_acc, f.w);
        }
      } else {
        part[(int64_t)leaf_part0[leaf] + (int64_t)kidx * nt + (ti - tb)] = v;
      }
    }
    __syncwarp();
  }
  }
  }
}

// Leaves whose near zone was split over 2 .. kP2PCombineWarp items (listed by
// the tree build): sum the items' partial sums in item order (deterministic),
// add the far field, write the outputs.
__global__ void __launch_bounds__(kThreads) k_p2p_combine(int64_t nsplit, const int *__restrict__ split,
                                                          const int *__restrict__ leaf_nitem,
                                                          const int *__restrict__ leaf_item0,
                                                          const int *__restrict__ item_t,
                                                          const int *__restrict__ leaf_part0,
                                                          const int *__restrict__ leaf_box,
                                                          const int *__restrict__ beg, const int *__restrict__ end,
                                                          const float4 *__restrict__ part,
                                                          const float4 *__restrict__ far,
                                                          const uint32_t *__restrict__ perm, float s1, float s2,
                                                          float *__restrict__ out_phi, float *__restrict__ out_acc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t si = (int64_t)blockIdx.x * kWarpsPerBlock + w;
  if (si >= nsplit) return;
  const int leaf = split[si];
  const int n = leaf_nitem[leaf];
  // complete sums already written, or a leaf for k_p2p_combine_big
  if (n <= 1 || n > kP2PCombineWarp || item_t[leaf_item0[leaf]] >= 0) return;
  const int box = leaf_box[leaf];
  const int tb = beg[box], nt = end[box] - tb;
  const float4 *pp = part + leaf_part0[leaf];
  for (int t = lane; t < nt; t += 32) {
    float sp = 0.f, cp = 0.f, sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f, sz = 0.f, cz = 0.f;
    for (int k = 0; k < n; ++k) {
      const float4 v = pp[(int64_t)k * nt + t];
      kahan_add(sp, cp, v.x);
      kahan_add(sx, cx, v.y);
      kahan_add(sy, cy, v.z);
      kahan_add(sz, cz, v.w);
    }
    const int ti = tb + t;
    const float4 f = far[ti];
    const uint32_t o = perm[ti];
    if (out_phi) out_phi[o] = fmaf(sp - cp, s1, f.x);
    if (out_acc) {
      out_acc[3 * (int64_t)o] = fmaf(sx - cx, s2, f.y);
      out_acc[3 * (int64_t)o + 1] = fmaf(sy - cy, s2, f.z);
      out_acc[3 * (int64_t)o + 2] = fmaf(sz - cz, s2, f.w);
    }
  }
}

__device__ __forceinline__ void two_sum_acc(float &s, float &e, float s2, float e2) {
  const float t = s + s2, bp = t - s;
  e = e + e2 + ((s - (t - bp)) + (s2 - bp));
  s = t;
}

// Leaves split over more than kP2PCombineWarp items (a small leaf beside
// large neighbour boxes, thousands of items): a block per leaf, a warp per
// target; the lanes take the items lane-strided (Kahan) and their sums meet
// in a fixed butterfly of two-sums (deterministic), lane 0 writing the output.
__global__ void __launch_bounds__(kThreads) k_p2p_combine_big(const int *__restrict__ big,
                                                              const int *__restrict__ leaf_nitem,
                                                              const int *__restrict__ leaf_part0,
                                                              const int *__restrict__ leaf_box,
                                                              const int *__restrict__ beg,
                                                              const int *__restrict__ end,
                                                              const float4 *__restrict__ part,
                                                              const float4 *__restrict__ far,
                                                              const uint32_t *__restrict__ perm, float s1, float s2,
                                                              float *__restrict__ out_phi,
                                                              float *__restrict__ out_acc) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int leaf = big[blockIdx.x];
  const int n = leaf_nitem[leaf];
  const int box = leaf_box[leaf];
  const int tb = beg[box], nt = end[box] - tb;
  const float4 *pp = part + leaf_part0[leaf];
  for (int t = w; t < nt; t += kWarpsPerBlock) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = lane; k < n; k += 32) {
      const float4 v = pp[(int64_t)k * nt + t];
      kahan_add(s[0], c[0], v.x);
      kahan_add(s[1], c[1], v.y);
      kahan_add(s[2], c[2], v.z);
      kahan_add(s[3], c[3], v.w);
    }
    float e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      e[q] = -c[q];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s[q], off), eo = __shfl_xor_sync(0xffffffffu, e[q], off);
        two_sum_acc(s[q], e[q], so, eo);
      }
    }
    if (lane == 0) {
      const int ti = tb + t;
      const float4 f = far[ti];
      const uint32_t o = perm[ti];
      if (out_phi) out_phi[o] = fmaf(s[0] + e[0], s1, f.x);
      if (out_acc) {
        out_acc[3 * (int64_t)o] = fmaf(s[1] + e[1], s2, f.y);
        out_acc[3 * (int64_t)o + 1] = fmaf(s[2] + e[2], s2, f.z);
        out_acc[3 * (int64_t)o + 2] = fmaf(s[3] + e[3], s2, f.w);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Green function transform, FP64. g(d) = g(h |d|_p) on the P^3 periodic grid,
// read from the level's lattice table gl[|d|_p^2] (gl[0] = g(unit offset)).
// g is real and even in every axis, so its transform is the separable cosine
// sum
//   G^(k) = sum_d g(d) cos(2 pi kx dx/P) cos(2 pi ky dy/P) cos(2 pi kz dz/P),
// real and even; only k in [0, P/2]^3 is stored.
__global__ void k_green_pass(int P, int pass, const double *__restrict__ gl, const double *__restrict__ in,
                             double *__restrict__ out) {
  const int H = P / 2 + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)H * H * H) return;
  const int a = (int)(i % H), b = (int)((i / H) % H), c = (int)(i / ((int64_t)H * H));
  // pass 0: a = kx, (b, c) = (|dy|, |dz|); pass 1: a = kx, b = ky, c = |dz|; pass 2: (a, b, c) = k
  const int k = pass == 0 ? a : (pass == 1 ? b : c);
  double s = 0.0;
  for (int d = 0; d < P; ++d) {
    const int dr = d <= P / 2 ? d : P - d;
    double v;
    if (pass == 0) {
      v = gl[dr * dr + b * b + c * c];
    } else if (pass == 1) {
      v = in[a + (int64_t)H * (dr + (int64_t)H * c)];
    } else {
      v = in[a + (int64_t)H * (b + (int64_t)H * dr)];
    }
    s += v * cospi(2.0 * (double)((k * d) % P) / (double)P);
  }
  out[i] = s;
}

// Green function transformed along x only (used by the x-transform / direct
// (y, z) convolution kernel): K[kx][a][b] = -(1/P) sum_{dx=0}^{P-1}
// (G(|dx|_p, a, b) - mean) cos(2 pi kx dx / P), FP64, stored FP32.
__global__ void k_green_kx(int P, int R, const double *__restrict__ gl, const float *__restrict__ mean, int level,
                           float *__restrict__ out) {
  const int H = P / 2 + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)H * R * R) return;
  const int b = (int)(i % R), a = (int)((i / R) % R), kx = (int)(i / ((int64_t)R * R));
  const double m = (double)mean[level];
  double s = 0.0;
  for (int d = 0; d < P; ++d) {
    const int dr = d <= P / 2 ? d : P - d;
    s += (gl[dr * dr + a * a + b * b] - m) * cospi(2.0 * (double)((kx * d) % P) / (double)P);
  }
  out[i] = (float)(-s / (double)P);
}

// Ng = 4 tables for the direct z sums: K2[kx][kyr][d] = sum_{kz=0}^{P-1}
// Gs(kx, kyr, |kz|_p) cos(2 pi kz d / P) with Gs = -G^/P^3 and Gs(0, 0, 0) = 0
// (the DC removal), from the FP64 transform of the reduced table `in`.
__global__ void k_green_kz(int P, int R, const double *__restrict__ in, float *__restrict__ out) {
  const int H = P / 2 + 1;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)H * H * R) return;
  const int d = (int)(i % R), kyr = (int)((i / R) % H), kx = (int)(i / ((int64_t)R * H));
  const double scale = -1.0 / ((double)P * P * P);
  double s = 0.0;
  for (int kz = 0; kz < P; ++kz) {
    const int kzr = kz <= P / 2 ? kz : P - kz;
    const double g = (kx == 0 && kyr == 0 && kzr == 0) ? 0.0 : scale * in[kx + (int64_t)H * (kyr + (int64_t)H * kzr)];
    s += g * cospi(2.0 * (double)((kz * d) % P) / (double)P);
  }
  out[i] = (float)s;
}

// Stores -G^/P^3 in FP32 with the DC term removed: G^(0)/P^3 is the mean m of
// G over the periodic grid, and convolving with G - m instead of G changes every
// output by the same constant m * sum(rho). That constant is added back to the
// target's local constant (it carries no force), while the FP32 transform no
// longer carries the large DC product, the dominant term of its round-off.
__global__ void k_green_store(int64_t n, const double *__restrict__ in, double scale, float *__restrict__ out,
                              float *__restrict__ mean_out, double inv_p3) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *mean_out = (float)(in[0] * inv_p3);
  if (i < n) out[i] = i == 0 ? 0.f : (float)(in[i] * scale);
}

// Packed-array gather and scatter of a batch of separately stored problems.
__device__ __forceinline__ int problem_of(const int64_t *off, int nprob, int64_t i) {
  int lo = 0, hi = nprob;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_batch_gather(const hpm_problem *__restrict__ desc, const int64_t *__restrict__ off, int nprob,
                               int64_t n, double *__restrict__ pos, double *__restrict__ mass) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = problem_of(off, nprob, i);
  const int64_t j = i - off[p];
  const double *src = desc[p].d_pos;
  pos[3 * i] = src[3 * j];
  pos[3 * i + 1] = src[3 * j + 1];
  pos[3 * i + 2] = src[3 * j + 2];
  mass[i] = desc[p].d_mass[j];
}

__global__ void k_batch_scatter(const hpm_problem *__restrict__ desc, const int64_t *__restrict__ off, int nprob,
                                int64_t n, const float *__restrict__ phi, const float *__restrict__ acc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = problem_of(off, nprob, i);
  const int64_t j = i - off[p];
  if (desc[p].d_phi) desc[p].d_phi[j] = phi[i];
  if (desc[p].d_acc) {
    desc[p].d_acc[3 * j] = acc[3 * i];
    desc[p].d_acc[3 * j + 1] = acc[3 * i + 1];
    desc[p].d_acc[3 * j + 2] = acc[3 * i + 2];
  }
}

}  // namespace

hpm_status precompute_green(hpm_plan_s *pl, cudaStream_t st) {
  HPM_TRY(build_lattice(pl, st));
  HPM_TRY(build_near_table(pl, st));
  const int P = 8 * pl->ng, H = P / 2 + 1;
  const int64_t h3 = (int64_t)H * H * H;
  const int D = pl->max_depth;
  pl->ghat_level_stride = h3;
  HPM_TRY(pl->ghat.ensure(sizeof(float) * h3 * (D + 1), st));
  HPM_CUDA(cudaMemsetAsync(pl->ghat.p, 0, sizeof(float) * h3 * (D + 1), st));
  HPM_TRY(pl->gmean.ensure(sizeof(float) * (D + 1), st));
  HPM_CUDA(cudaMemsetAsync(pl->gmean.p, 0, sizeof(float) * (D + 1), st));
  double *a = nullptr, *b = nullptr;
  HPM_TRY(lib_malloc_async((void **)&a, sizeof(double) * h3, st));
  HPM_TRY(lib_malloc_async((void **)&b, sizeof(double) * h3, st));
  const double scale = -1.0 / ((double)P * P * P);
  if (pl->ng == 4) {
    pl->kz_green_stride = (int64_t)H * H * (4 * pl->ng);
    HPM_TRY(pl->kz_green.ensure(sizeof(float) * pl->kz_green_stride * (D + 1), st));
    HPM_CUDA(cudaMemsetAsync(pl->kz_green.p, 0, sizeof(float) * pl->kz_green_stride * (D + 1), st));
  }
  for (int l = 2; l <= D; ++l) {
    const double *gl = pl->glat.as<double>() + pl->glat_stride * l;
    k_green_pass<<<blocks_for(h3), kThreads, 0, st>>>(P, 0, gl, nullptr, a);
    HPM_LAUNCHED((int64_t *)nullptr);
    k_green_pass<<<blocks_for(h3), kThreads, 0, st>>>(P, 1, gl, a, b);
    HPM_LAUNCHED((int64_t *)nullptr);
    k_green_pass<<<blocks_for(h3), kThreads, 0, st>>>(P, 2, gl, b, a);
    HPM_LAUNCHED((int64_t *)nullptr);
    k_green_store<<<blocks_for(h3), kThreads, 0, st>>>(h3, a, scale, pl->ghat.as<float>() + h3 * l,
                                                       pl->gmean.as<float>() + l, -scale);
    HPM_LAUNCHED((int64_t *)nullptr);
    if (pl->ng == 4) {
      k_green_kz<<<blocks_for(pl->kz_green_stride), kThreads, 0, st>>>(
          P, 4 * pl->ng, a, pl->kz_green.as<float>() + pl->kz_green_stride * l);
      HPM_LAUNCHED((int64_t *)nullptr);
    }
  }
  HPM_CUDA(cudaFreeAsync(a, st));
  HPM_CUDA(cudaFreeAsync(b, st));
  // x-transformed tables for the orders the x-transform kernel serves
  if (pl->ng == 2 || pl->ng == 3 || pl->ng == 4 || pl->ng == 5 || pl->ng == 6) {
    const int R = 4 * pl->ng;
    pl->kx_green_stride = (int64_t)H * R * R;
    HPM_TRY(pl->kx_green.ensure(sizeof(float) * pl->kx_green_stride * (D + 1), st));
    HPM_CUDA(cudaMemsetAsync(pl->kx_green.p, 0, sizeof(float) * pl->kx_green_stride * (D + 1), st));
    for (int l = 2; l <= D; ++l) {
      k_green_kx<<<blocks_for(pl->kx_green_stride), kThreads, 0, st>>>(
          P, R, pl->glat.as<double>() + pl->glat_stride * l, pl->gmean.as<float>(), l,
          pl->kx_green.as<float>() + pl->kx_green_stride * l);
      HPM_LAUNCHED((int64_t *)nullptr);
    }
  }
  return HPM_OK;
}

hpm_status batch_gather(const hpm_problem *d_desc, const int64_t *d_off, int nprob, int64_t n, double *pos,
                        double *mass, cudaStream_t st) {
  if (n <= 0) return HPM_OK;
  k_batch_gather<<<blocks_for(n), kThreads, 0, st>>>(d_desc, d_off, nprob, n, pos, mass);
  HPM_LAUNCHED((int64_t *)nullptr);
  return HPM_OK;
}

hpm_status batch_scatter(const hpm_problem *d_desc, const int64_t *d_off, int nprob, int64_t n, const float *phi,
                         const float *acc, cudaStream_t st) {
  if (n <= 0) return HPM_OK;
  k_batch_scatter<<<blocks_for(n), kThreads, 0, st>>>(d_desc, d_off, nprob, n, phi, acc);
  HPM_LAUNCHED((int64_t *)nullptr);
  return HPM_OK;
}

static LevelTable make_levels(const hpm_plan_s *pl) {
  LevelTable lt{};
  lt.nlev = pl->max_depth + 1;
  for (int l = 0; l <= pl->max_depth + 1; ++l) lt.off[l] = pl->lvl_off[l];
  return lt;
}

static void record(hpm_plan_s *pl, int i, cudaStream_t st) {
  if (pl->events_ready) cudaEventRecord(pl->ev[i], st);
}

hpm_status solve(hpm_plan_s *pl, const double *d_pos, const double *d_mass, float *d_phi, float *d_acc,
                 cudaStream_t st) {
  TreeDev &t = pl->t;
  SolveDev &s = pl->s;
  const int64_t n = pl->n;
  int64_t launches = 0;
  pl->stats.m2l_launches = 0;
  pl->stats.m2l_targets = pl->ntgt;
  pl->stats.m2l_parents = 0;
  pl->stats.ms_m2l_kernel = 0.f;
  pl->stats.p2p_pairs = pl->npairs;
  if (n == 0) return HPM_OK;
  const int ng = pl->ng, m3 = ng * ng * ng;
  // target (local) gridlets: Ng^3 nodes, or (Ng + 2)^3 widened (Sec. 2.5)
  const int ngl = pl->ng_loc, m3l = ngl * ngl * ngl;
  const int D = pl->max_depth;
  const int64_t off2 = D >= 2 ? pl->lvl_off[2] : pl->nbox;
  const int64_t nrow = pl->nbox - off2;
  HPM_TRY(t.spm.ensure(2 * sizeof(float4) * n, st));
  HPM_TRY(s.grid.ensure(sizeof(float) * m3 * (nrow > 0 ? nrow : 1), st));
  HPM_TRY(s.loc.ensure(sizeof(float) * m3l * (pl->ntgt > 0 ? pl->ntgt : 1), st));
  HPM_TRY(s.m2l_raw.ensure(sizeof(float) * m3l * (pl->ntgt > 0 ? pl->ntgt : 1), st));
  HPM_TRY(s.locc.ensure(sizeof(float) * (pl->ntgt > 0 ? pl->ntgt : 1), st));
  HPM_TRY(s.m2lc.ensure(sizeof(float) * (pl->ntgt > 0 ? pl->ntgt : 1), st));
  HPM_TRY(s.far.ensure(sizeof(float4) * n, st));
  float4 *hi = t.spm.as<float4>();
  float4 *lo = hi + n;
  const LevelTable lt = make_levels(pl);
  const double *o = pl->dom.origin;

  record(pl, 0, st);
  const bool unit = o[0] == 0.0 && o[1] == 0.0 && o[2] == 0.0 && pl->dom.side == 1.0;
  (unit ? k_gather<true> : k_gather<false>)<<<blocks_for(n), kThreads, 0, st>>>(
      n, t.perm.as<uint32_t>(), d_pos, d_mass, o[0], o[1], o[2], 1.0 / pl->dom.side, hi, lo);
  HPM_LAUNCHED(&launches);
  record(pl, 1, st);
  // the dense source-to-target kernel's per-(problem, level) scales, taken
  // as the P2G and child-to-parent kernels write the rows
  int *amax = nullptr;
  const int nlev = D + 1;
  if (use_tc_m2l(pl) && nrow > 0) {
    const size_t nslot = (size_t)(pl->nprob > 0 ? pl->nprob : 1) * nlev;
    HPM_TRY(s.level_amax.ensure(sizeof(int) * nslot, st));
    HPM_CUDA(cudaMemsetAsync(s.level_amax.p, 0, sizeof(int) * nslot, st));
    amax = s.level_amax.as<int>();
  }
  if (pl->np2g) {
    auto kp = ng == 4 ? k_p2g<4> : k_p2g<0>;
    kp<<<warp_blocks(pl->np2g), kThreads, 0, st>>>(pl->np2g, t.p2g_box.as<int>(), lt, pl->tab,
                                                   t.box_key.as<uint64_t>(), t.box_beg.as<int>(),
                                                   t.box_end.as<int>(), hi, lo, off2,
                                                   s.grid.as<float>(), amax, nlev);
    HPM_LAUNCHED(&launches);
  }
  record(pl, 2, st);
  for (int l = pl->depth_reached - 1; l >= 2; --l) {
    const int64_t b = pl->lvl_off[l], e = pl->lvl_off[l + 1];
    if (e <= b) continue;
    if (ng == 4) {
      const int W = gridlet_warps(pl);
      auto km = W == 2 ? k_m2m4<2> : (W == 4 ? k_m2m4<4> : k_m2m4<8>);
      km<<<(unsigned)((e - b + W - 1) / W), W * 32, 0, st>>>(b, e, pl->tab, t.box_flags.as<uint8_t>(),
                                                            t.box_child.as<int>(), off2, s.grid.as<float>(),
                                                            t.box_key.as<uint64_t>(), l, amax, nlev);
    } else
      k_m2m<<<gwarp_blocks(e - b), kGThreads, 0, st>>>(b, e, pl->tab, t.box_flags.as<uint8_t>(),
                                                     t.box_child.as<int>(), off2, s.grid.as<float>(),
                                                     t.box_key.as<uint64_t>(), l, amax, nlev);
    HPM_LAUNCHED(&launches);
  }
  record(pl, 3, st);
  if (pl->ntgt) {
    int64_t ml = 0;
    HPM_TRY(launch_m2l(pl, st, &ml));
    launches += ml;
    pl->stats.m2l_launches = ml;
  }
  record(pl, 4, st);
  for (int l = 2; l <= pl->depth_reached; ++l) {
    const int64_t b = pl->tgt_lvl_off[l], e = pl->tgt_lvl_off[l + 1];
    if (e <= b) continue;
    if (ngl == 4) {
      const int W = gridlet_warps(pl);
      auto kl = W == 2 ? k_l2l4<2> : (W == 4 ? k_l2l4<4> : k_l2l4<8>);
      kl<<<(unsigned)((e - b + W - 1) / W), W * 32, 0, st>>>(
          b, e, l, pl->tab_loc, t.tgt_box.as<int>(), t.box_tgt.as<int>(), t.box_parent.as<int>(),
          t.box_key.as<uint64_t>(), s.m2l_raw.as<float>(), s.loc.as<float>(), s.locc.as<float>(),
          s.m2lc.as<float>());
    } else
      k_l2l_df<<<(unsigned)((e - b + kDfWarps - 1) / kDfWarps), 32 * kDfWarps, 0, st>>>(
          b, e, l, pl->tab_loc, t.tgt_box.as<int>(), t.box_tgt.as<int>(), t.box_parent.as<int>(),
          t.box_key.as<uint64_t>(), s.m2l_raw.as<float>(), s.loc.as<float>(), s.locc.as<float>(),
          s.m2lc.as<float>());
    HPM_LAUNCHED(&launches);
  }
  record(pl, 5, st);
  auto kg = ngl == 4 ? k_g2p<4> : (ngl == 6 ? k_g2p_df<6> : k_g2p_df<0>);
  kg<<<blocks_for(n), kThreads, 0, st>>>(n, t.pbox.as<int>(), t.box_tgt.as<int>(), lt, pl->tab_loc,
                                            (float)(1.0 / pl->dom.side), t.box_key.as<uint64_t>(), hi, lo,
                                            s.loc.as<float>(), s.locc.as<float>(), s.far.as<float4>());
  HPM_LAUNCHED(&launches);
  record(pl, 6, st);
  {
    // pairs are summed in unit-cube coordinates (eps / S, lambda / S); the
    // closed forms are scaled back by 1/S (potential) and 1/S^2 (acceleration)
    // once per target, the user kernel's table is in physical units already
    const double S = pl->dom.side;
    const double eu = pl->green.eps / S;
    const int kind = pl->green.kind == HPM_GREEN_USER ? 2 : (pl->green.kind == HPM_GREEN_YUKAWA ? 1 : 0);
    NearKernel nk{};
    nk.eps2 = kind == 2 ? 0.f : (float)(eu * eu);
    nk.inv_lambda = kind == 1 ? (float)(S / pl->green.lambda) : 0.f;
    nk.tab = pl->near_tab.as<float4>();
    const float s1 = kind == 2 ? 1.f : (float)(1.0 / S), s2 = kind == 2 ? 1.f : (float)(1.0 / (S * S));
    HPM_TRY(s.part.ensure(sizeof(float4) * (pl->npart > 0 ? pl->npart : 1), st));
    auto kp = kind == 0 ? k_p2p<0> : (kind == 1 ? k_p2p<1> : k_p2p<2>);
    static DeviceCache p2p_cache[3];
    int p2p_resident = 1;
    HPM_TRY(device_cached(p2p_cache[kind], [kp](int *v) -> hpm_status {
      HPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(v, kp, kThreads, 0));
      if (*v < 1) *v = 1;
      return HPM_OK;
    }, &p2p_resident));
    HPM_TRY(s.work.ensure(sizeof(unsigned long long), st));
    HPM_CUDA(cudaMemsetAsync(s.work.p, 0, sizeof(unsigned long long), st));
    const unsigned p2p_grid = (unsigned)std::min<int64_t>(warp_blocks(pl->nitem), (int64_t)p2p_resident * sm_count());
    kp<<<p2p_grid, kThreads, 0, st>>>(
        pl->nitem, t.item_leaf.as<int>(), t.item_s0.as<int>(), t.item_s1.as<int>(), t.item_t.as<int>(),
        t.leaf_nitem.as<int>(),
        t.leaf_item0.as<int>(), t.leaf_part0.as<int>(), t.leaf_box.as<int>(), t.box_nb.as<int>(),
        t.box_beg.as<int>(), t.box_end.as<int>(), hi, lo, s.far.as<float4>(), t.perm.as<uint32_t>(),
        t.box_key.as<uint64_t>(), lt, nk, s1, s2, d_phi, d_acc, s.part.as<float4>(),
        s.work.as<unsigned long long>());
    HPM_LAUNCHED(&launches);
    if (pl->nsplit > 0) {
      k_p2p_combine<<<warp_blocks(pl->nsplit), kThreads, 0, st>>>(
          pl->nsplit, t.split_leaf.as<int>(), t.leaf_nitem.as<int>(), t.leaf_item0.as<int>(), t.item_t.as<int>(), t.leaf_part0.as<int>(), t.leaf_box.as<int>(), t.box_beg.as<int>(),
          t.box_end.as<int>(), s.part.as<float4>(), s.far.as<float4>(), t.perm.as<uint32_t>(), s1, s2, d_phi,
          d_acc);
      HPM_LAUNCHED(&launches);
    }
    if (pl->nbig > 0) {
      k_p2p_combine_big<<<(unsigned)pl->nbig, kThreads, 0, st>>>(
          t.big_leaf.as<int>(), t.leaf_nitem.as<int>(), t.leaf_part0.as<int>(), t.leaf_box.as<int>(),
          t.box_beg.as<int>(), t.box_end.as<int>(), s.part.as<float4>(), s.far.as<float4>(),
          t.perm.as<uint32_t>(), s1, s2, d_phi, d_acc);
      HPM_LAUNCHED(&launches);
    }
  }
  record(pl, 7, st);
  pl->stats.launches += launches;
  return HPM_OK;
}

}  // namespace hpm

extern "C" hpm_status hpm_check_conversions(const double *d_in, int64_t n_d, const float *f_in, int64_t n_f,
                                            int64_t *mismatches, void *stream) {
  if (!mismatches || n_d < 0 || n_f < 0 || (n_d > 0 && !d_in) || (n_f > 0 && !f_in)) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  hpm::DevBuf cnt;
  HPM_TRY(cnt.ensure(sizeof(unsigned long long), st));
  hpm_status s = HPM_OK;
  cudaError_t e = cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), st);
  const int64_t n = std::max(n_d, n_f);
  if (e == cudaSuccess && n > 0) {
    hpm::k_check_conversions<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_in, n_d, f_in, n_f,
                                                                          cnt.as<unsigned long long>());
    e = cudaGetLastError();
  }
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    hpm::set_cuda_error(e);
    s = HPM_ERR_CUDA;
  }
  cnt.release(st);
  cudaStreamSynchronize(st);
  *mismatches = (int64_t)h;
  return s;
}
