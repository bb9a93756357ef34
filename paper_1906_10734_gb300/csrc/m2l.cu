// Source-to-target transformation (Sec. 2.1): for every target cell t at level
// l >= 2, the effective masses of the 6^3 level-l boxes around t's parent
// (zero where a box is empty, outside the domain or in t's near zone) form a
// (6 Ng)^3 grid that is zero padded to P^3 = (8 Ng)^3 and convolved with the
// exact Green function by one FFT; the Ng^3 values at t's gridlet nodes are
// kept.
//
// The convolution is periodic with period P, so the block may be placed at
// any circular offset. Both kernels here place it so that the target's nodes
// sit at FFT positions 0 .. Ng-1: the Green transform then needs no phase
// factor per child parity (one real table per level serves all 8 parities)
// and the inverse transform is pruned to those Ng outputs per axis.
#include <cmath>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

struct Levels {
  int64_t off[kMaxDepth + 3];
  int nlev;
};

__device__ __forceinline__ int level_of(const Levels &lt, int64_t box) {
  int l = 0;
  while (l + 1 < lt.nlev && lt.off[l + 1] <= box) ++l;
  return l;
}

struct TreeRefs {
  const float *grid;
  float *out;
  float *outc;          // per target: -mean(G) * sum(rho), the constant part
  const float *gmean;   // per level: mean of G over the periodic grid
  const int *tgt_box;
  const int *parent;
  const int *nb;
  const int *child;
  const uint64_t *key;
  const float *ghat;
  int64_t ghat_stride;
  int64_t off2;
  int64_t ntgt;
};

// Block table of one target: row of each of the 216 boxes, -1 where the box
// is empty, outside the domain or within Chebyshev distance 1 of the target.
__device__ __forceinline__ void fill_block(const TreeRefs &r, int box, int tx, int ty, int tz, int *blk) {
  const int p = r.parent[box];
  for (int j = threadIdx.x; j < 216; j += blockDim.x) {
    const int bx = j % 6, by = (j / 6) % 6, bz = j / 36;
    int row = -1;
    const int cheb = max(abs(bx - tx), max(abs(by - ty), abs(bz - tz)));
    if (cheb >= 2) {
      const int q = r.nb[(int64_t)p * 27 + (bx >> 1) + 3 * (by >> 1) + 9 * (bz >> 1)];
      if (q >= 0) {
        const int c = r.child[(int64_t)q * 8 + (bx & 1) + 2 * (by & 1) + 4 * (bz & 1)];
        if (c >= 0) row = (int)(c - r.off2);
      }
    }
    blk[j] = row;
  }
}

// ===========================================================================
// Fast path, Ng = 4 (P = 32).
// ===========================================================================
namespace f4 {
constexpr int kP = 32, kB = 24, kH = 17;
constexpr int kLS = 25;                // line stride of the x-pass output [z][y]
constexpr int kYS = 33;                // line stride of the y-pass output [z][ky]
constexpr int kSlab = kB * kYS;        // float2 per kx slab (>= 24 * 25)
constexpr int kThreads = 288;          // 9 warps; 288 line pairs in the x pass
constexpr int kWarps = kThreads / 32;
constexpr size_t kSmem = sizeof(float2) * kH * kSlab + sizeof(int) * 216 + sizeof(float) * kH * 32 +
                         sizeof(float2) * 32 + 16;

struct Params {
  float2 w[kP];  // w[e] = exp(-2 pi i e / 32)
  TreeRefs r;
  Levels lt;
  const float *kz;   // z-transformed Green tables, kz_stride floats per level
  int64_t kz_stride;
  const int *tblk;   // per target: 216 source rows (interaction zone), -1 = none
  const int *tinfo;  // per target: level << 3 | child octant
};

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

constexpr int brev5(int i) {
  return ((i & 1) << 4) | ((i & 2) << 2) | (i & 4) | ((i & 8) >> 2) | ((i & 16) >> 4);
}

// In-register radix-2 decimation-in-time FFT of 32 points.
// SIGN = -1: forward (w), SIGN = +1: backward (conj w). Unnormalised.
template <int SIGN>
__device__ __forceinline__ void fft32(float2 (&a)[32], const float2 (&w)[kP]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int j = brev5(i);
    if (j > i) {
      const float2 t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < 32; half <<= 1) {
#pragma unroll
    for (int i = 0; i < 32; i += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const int e = k * (16 / half);
        float2 v = a[i + k + half];
        if (e == 8) {
          v = SIGN < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
        } else if (e != 0) {
          float2 wv = w[e];
          if (SIGN > 0) wv.y = -wv.y;
          v = cmul(v, wv);
        }
        const float2 u = a[i + k];
        a[i + k] = cadd(u, v);
        a[i + k + half] = csub(u, v);
      }
    }
  }
}

// x pass: two real x-lines (y0, y0+1) at height z as one complex FFT, block
// placed so that the target's x nodes land at 0..3. Writes 2x the spectra
// (the 1/2 of the two-for-one split is applied at the end).
template <int TX>
__device__ __forceinline__ void pass_x(const Params &pr, const int *blk, float2 *X) {
  const int t = threadIdx.x;
  const int z = t / 12, y0 = 2 * (t % 12);
  const int bz = z >> 2, kz = z & 3, by = y0 >> 2, ky0 = y0 & 3;
  float2 a[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) a[i] = make_float2(0.f, 0.f);
#pragma unroll
  for (int bx = 0; bx < 6; ++bx) {
    const int slot = (bx - TX) & 7;
    const int row = blk[bx + 6 * by + 36 * bz];
    if (row >= 0) {
      const float *g = pr.r.grid + (int64_t)row * 64 + 16 * kz + 4 * ky0;
      const float4 v0 = __ldg(reinterpret_cast<const float4 *>(g));
      const float4 v1 = __ldg(reinterpret_cast<const float4 *>(g + 4));
      a[4 * slot + 0] = make_float2(v0.x, v1.x);
      a[4 * slot + 1] = make_float2(v0.y, v1.y);
      a[4 * slot + 2] = make_float2(v0.z, v1.z);
      a[4 * slot + 3] = make_float2(v0.w, v1.w);
    }
  }
  fft32<-1>(a, pr.w);
#pragma unroll
  for (int k = 0; k <= 16; ++k) {
    const float2 zk = a[k], zm = a[(32 - k) & 31];
    X[k * kSlab + z * kLS + y0] = make_float2(zk.x + zm.x, zk.y - zm.y);
    X[k * kSlab + z * kLS + y0 + 1] = make_float2(zk.y + zm.y, zm.x - zk.x);
  }
}

// y pass, direct z sums with the z-transformed Green table, pruned inverse y,
// for one kx slab (one warp).
template <int N0Z>
__device__ __forceinline__ void pass_slab(const Params &pr, int kx, int n0y, float2 *slab, const float *kz,
                                          const float2 *tw, float *V, float *dc) {
  const int lane = threadIdx.x & 31;
  float2 a[32];
  // y pass: lane = z
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    const int u = (r + n0y) & 31;
    a[r] = (lane < kB && u < kB) ? slab[lane * kLS + u] : make_float2(0.f, 0.f);
  }
  fft32<-1>(a, pr.w);
  __syncwarp();
  if (lane < kB) {
#pragma unroll
    for (int r = 0; r < 32; ++r) slab[lane * kYS + r] = a[r];
  }
  __syncwarp();
  // z: the forward transform, the Green product and the inverse pruned to the
  // target's 4 planes are one linear map from the 24 block planes, evaluated
  // as direct sums with the Green transform inverse-transformed along z,
  // W(z') = sum_u Y(u) K2[kx][|ky|][|N0Z + z' - u|] (lane = ky)
  float2 W0 = make_float2(0.f, 0.f), W1 = W0, W2 = W0, W3 = W0;
  {
    const int kyr = lane <= 16 ? lane : 32 - lane;
    const float *krow = kz + (kx * kH + kyr) * 16;
    float k[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) k[d] = __ldg(krow + d);
    float dsum = 0.f;
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const float2 v = slab[u * kYS + lane];
      dsum += v.x;
      const int a0 = N0Z - u, a1 = N0Z + 1 - u, a2 = N0Z + 2 - u, a3 = N0Z + 3 - u;  // constant after unrolling
      const float k0 = k[a0 < 0 ? -a0 : a0], k1 = k[a1 < 0 ? -a1 : a1], k2 = k[a2 < 0 ? -a2 : a2],
                  k3 = k[a3 < 0 ? -a3 : a3];
      W0.x = fmaf(v.x, k0, W0.x); W0.y = fmaf(v.y, k0, W0.y);
      W1.x = fmaf(v.x, k1, W1.x); W1.y = fmaf(v.y, k1, W1.y);
      W2.x = fmaf(v.x, k2, W2.x); W2.y = fmaf(v.y, k2, W2.y);
      W3.x = fmaf(v.x, k3, W3.x); W3.y = fmaf(v.y, k3, W3.y);
    }
    if (kx == 0 && lane == 0) *dc = 0.5f * dsum;  // sum of the block (x pass doubles)
  }
  // inverse over ky for y' = 0..3: products, then a transposed warp reduction
  const float2 Wz[4] = {W0, W1, W2, W3};
  float v[32];
#pragma unroll
  for (int yy = 0; yy < 4; ++yy) {
    const float2 t = tw[(lane * yy) & 31];  // e^{+2 pi i ky y'/32}
#pragma unroll
    for (int zz = 0; zz < 4; ++zz) {
      const float2 pz = yy == 0 ? Wz[zz] : cmul(Wz[zz], t);
      v[2 * (yy + 4 * zz)] = pz.x;
      v[2 * (yy + 4 * zz) + 1] = pz.y;
    }
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = upper ? v[i] : v[i + s];
      const float keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  V[kx * 32 + lane] = v[0];
}

__global__ void __launch_bounds__(kThreads, 2) k_m2l4(const __grid_constant__ Params pr) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2 *X = reinterpret_cast<float2 *>(smem);
  int *blk = reinterpret_cast<int *>(X + kH * kSlab);
  float *V = reinterpret_cast<float *>(blk + 216);
  float2 *tw = reinterpret_cast<float2 *>(V + kH * 32);
  float *dc = reinterpret_cast<float *>(tw + 32);
  if (threadIdx.x < 32) tw[threadIdx.x] = make_float2(pr.w[threadIdx.x].x, -pr.w[threadIdx.x].y);
  const int warp = threadIdx.x >> 5;
  // the next target's interaction-zone rows and (level, octant) are loaded one
  // target ahead, so no dependent global load stalls the CTA between targets
  int pre_row = -1, pre_info = 0;
  if (blockIdx.x < pr.r.ntgt) {
    if (threadIdx.x < 216) pre_row = __ldg(pr.tblk + (int64_t)blockIdx.x * 216 + threadIdx.x);
    pre_info = __ldg(pr.tinfo + blockIdx.x);
  }
  for (int64_t t = blockIdx.x; t < pr.r.ntgt; t += gridDim.x) {
    if (threadIdx.x < 216) blk[threadIdx.x] = pre_row;
    const int info = pre_info;
    const int oc = info & 7, lev = info >> 3;
    const int tx = 2 + (oc & 1), ty = 2 + ((oc >> 1) & 1), tz = 2 + ((oc >> 2) & 1);
    const float *kzt = pr.kz + pr.kz_stride * lev;
    const int64_t tn = t + gridDim.x;
    if (tn < pr.r.ntgt) {
      if (threadIdx.x < 216) pre_row = __ldg(pr.tblk + tn * 216 + threadIdx.x);
      pre_info = __ldg(pr.tinfo + tn);
    }
    __syncthreads();
    if (tx == 2) pass_x<2>(pr, blk, X);
    else pass_x<3>(pr, blk, X);
    __syncthreads();
    for (int kx = warp; kx < kH; kx += kWarps) {
      if (tz == 2) pass_slab<8>(pr, kx, 4 * ty, X + kx * kSlab, kzt, tw, V, dc);
      else pass_slab<12>(pr, kx, 4 * ty, X + kx * kSlab, kzt, tw, V, dc);
    }
    __syncthreads();
    if (threadIdx.x == 64) pr.r.outc[t] = -pr.r.gmean[lev] * *dc;
    if (threadIdx.x < 64) {
      const int p = threadIdx.x;
      const int xx = p & 3, yz = p >> 2;  // yz = y' + 4 z'
      float s = 0.f;
#pragma unroll
      for (int kx = 0; kx < kH; ++kx) {
        const float2 vv = make_float2(V[kx * 32 + 2 * yz], V[kx * 32 + 2 * yz + 1]);
        const float2 t2 = tw[(kx * xx) & 31];
        const float re = vv.x * t2.x - vv.y * t2.y;
        s += (kx == 0 || kx == 16) ? re : 2.f * re;
      }
      pr.r.out[t * 64 + p] = 0.5f * s;
    }
  }
}
}  // namespace f4

// ===========================================================================
// Orders 2, 3, 5, 6: one CTA per parent cell, the parent's whole (6 Ng)^3
// block of effective masses resident in shared memory. For each kx in
// [0, P/2] the x-lines of the block are transformed once (a DFT along x shared
// by the parent's children); each child then takes its near-zone-masked copy
// of those spectra and convolves them directly over (y, z) with the Green
// function transformed along x, K[kx][|dy|][|dz|] (exact: every
// interaction-zone offset is below P/2 in each axis); the target values
// accumulate over kx in registers. This is the periodic convolution of
// Sec. 2.1 evaluated with the transform along one axis only, which at these
// sizes costs about the nominal FFT count and needs no (8 Ng)^3 spectrum on chip.
// ===========================================================================
namespace xd {
// threads per CTA and CTAs per SM for each order (the block takes 12, 33, 73,
// 136 and 230 KB of shared memory for Ng = 2, 3, 4, 5, 6)
template <int NG> struct Launch { static constexpr int threads = 512, min_blocks = 1; };
template <> struct Launch<2> { static constexpr int threads = 256, min_blocks = 2; };
template <> struct Launch<3> { static constexpr int threads = 256, min_blocks = 2; };
template <> struct Launch<4> { static constexpr int threads = 256, min_blocks = 2; };

struct Params {
  TreeRefs r;
  Levels lt;
  const int *par_box;
  const int *box_tgt;
  int64_t npar;
  const float *kxg;
  int64_t kx_stride;
};

template <int NG>
struct Geo {
  static constexpr int B = 6 * NG, BP = B + 1, P = 8 * NG, H = P / 2 + 1, R = 4 * NG, M3 = NG * NG * NG;
  static constexpr int N2 = 3 * NG;  // near range of a child along one axis
  static constexpr size_t kRho = (size_t)B * B * BP, kX = (size_t)B * B, kXn = 2 * (size_t)N2 * N2,
                          kPart = 2 * (size_t)NG * B * NG;
  static constexpr size_t kSmem = sizeof(float) * kRho + sizeof(float2) * (kX + kXn + kPart + B) +
                                  sizeof(float) * 216 + sizeof(int) * (216 + 32);
};

// Partial sums over zs for one (child, y', ys): acc[z'] = sum_zs Xc(ys, zs) K[dy][|Zt + z' - zs|].
template <int NG, int TZ>
__device__ __forceinline__ void conv_row(const float2 *__restrict__ X, const float2 *__restrict__ Xn, int ys,
                                         bool ynear, int ybase, const float *__restrict__ krow_g,
                                         float2 *__restrict__ out) {
  using G = Geo<NG>;
  float kr[G::R];
#pragma unroll
  for (int d = 0; d < G::R; ++d) kr[d] = __ldg(krow_g + d);
  float2 acc[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
  for (int zs = 0; zs < G::B; ++zs) {
    constexpr int zlo = NG * (TZ - 1), zhi = NG * (TZ + 2);
    const bool znear = zs >= zlo && zs < zhi;
    const float2 xv = (znear && ynear) ? Xn[(ys - ybase) * G::N2 + (zs - zlo)] : X[zs * G::B + ys];
#pragma unroll
    for (int q = 0; q < NG; ++q) {
      const int dz = NG * TZ + q - zs;
      const float k = kr[dz < 0 ? -dz : dz];
      acc[q].x = fmaf(xv.x, k, acc[q].x);
      acc[q].y = fmaf(xv.y, k, acc[q].y);
    }
  }
#pragma unroll
  for (int q = 0; q < NG; ++q) out[q] = acc[q];
}

template <int NG>
__global__ void __launch_bounds__(Launch<NG>::threads, Launch<NG>::min_blocks)
    k_m2l_xdft(const __grid_constant__ Params pr) {
  using G = Geo<NG>;
  constexpr int B = G::B, BP = G::BP, P = G::P, H = G::H, R = G::R, M3 = G::M3, N2 = G::N2;
  extern __shared__ __align__(16) unsigned char smem[];
  float *rho = reinterpret_cast<float *>(smem);
  float2 *X = reinterpret_cast<float2 *>(rho + G::kRho);
  float2 *Xn = X + G::kX;
  float2 *part = Xn + G::kXn;
  float2 *tw = part + G::kPart;
  float *boxsum = reinterpret_cast<float *>(tw + B);
  int *blk = reinterpret_cast<int *>(boxsum + 216);
  int *kid = blk + 216;  // [0..7]: child box, [8..15]: target index, [16]: count
  const int tid = threadIdx.x;
  for (int64_t pi = blockIdx.x; pi < pr.npar; pi += gridDim.x) {
    const int p = pr.par_box[pi];
    // children (targets) and the unmasked 6^3 block of level-(l) boxes
    if (tid == 0) {
      int n = 0;
      for (int o = 0; o < 8; ++o) {
        const int c = pr.r.child[(int64_t)p * 8 + o];
        if (c >= 0) {
          kid[n] = c;
          kid[8 + n] = pr.box_tgt[c];
          ++n;
        }
      }
      kid[16] = n;
    }
    for (int j = tid; j < 216; j += blockDim.x) {
      const int bx = j % 6, by = (j / 6) % 6, bz = j / 36;
      int row = -1;
      const int q = pr.r.nb[(int64_t)p * 27 + (bx >> 1) + 3 * (by >> 1) + 9 * (bz >> 1)];
      if (q >= 0) {
        const int c = pr.r.child[(int64_t)q * 8 + (bx & 1) + 2 * (by & 1) + 4 * (bz & 1)];
        if (c >= 0) row = (int)(c - pr.r.off2);
      }
      blk[j] = row;
    }
    __syncthreads();
    const int nkid = kid[16];
    if (nkid == 0) {
      __syncthreads();
      continue;
    }
    const int lev = level_of(pr.lt, kid[0]);
    const float *K = pr.kxg + pr.kx_stride * lev;
    for (int64_t idx = tid; idx < (int64_t)B * B * B; idx += blockDim.x) {
      const int x = (int)(idx % B), y = (int)((idx / B) % B), z = (int)(idx / (B * B));
      const int row = blk[x / NG + 6 * (y / NG) + 36 * (z / NG)];
      rho[((int64_t)z * B + y) * BP + x] =
          row >= 0 ? __ldg(pr.r.grid + (int64_t)row * M3 + (x % NG) + NG * ((y % NG) + NG * (z % NG))) : 0.f;
    }
    for (int j = tid; j < 216; j += blockDim.x) {
      float s = 0.f;
      if (blk[j] >= 0)
        for (int e = 0; e < M3; ++e) s += __ldg(pr.r.grid + (int64_t)blk[j] * M3 + e);
      boxsum[j] = s;
    }
    // owner of Phi(kid, y', z', x' = 0..NG-1) across the kx loop
    const bool owner = tid < nkid * NG * NG;
    const int ok = tid / (NG * NG), oy = (tid / NG) % NG, oz = tid % NG;
    int otx = 0;
    if (owner) otx = 2 + (int)(pr.r.key[kid[ok]] & 1u);
    float phi[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) phi[q] = 0.f;
    for (int kx = 0; kx < H; ++kx) {
      __syncthreads();  // rho ready / previous kx done with X, Xn, part, tw
      for (int x = tid; x < B; x += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)((kx * x) % P) / (float)P, &s, &c);
        tw[x] = make_float2(c, s);
      }
      __syncthreads();
      // DFT along x of every line, shared by the children
      for (int line = tid; line < B * B; line += blockDim.x) {
        const int y = line % B, z = line / B;
        const float *rr = rho + ((int64_t)z * B + y) * BP;
        float2 s = make_float2(0.f, 0.f);
#pragma unroll 6
        for (int x = 0; x < B; ++x) {
          s.x = fmaf(rr[x], tw[x].x, s.x);
          s.y = fmaf(rr[x], tw[x].y, s.y);
        }
        X[z * B + y] = s;
      }
      const float *Kk = K + (int64_t)kx * R * R;
      const float wk = (kx == 0 || 2 * kx == P) ? 1.f : 2.f;
      for (int k0 = 0; k0 < nkid; k0 += 2) {
        const int nk = min(2, nkid - k0);
        __syncthreads();  // X complete; previous pair done with Xn, part
        // near-zone masked lines of each child: subtract the masked boxes' part
        for (int e = tid; e < nk * N2 * N2; e += blockDim.x) {
          const int s = e / (N2 * N2), yl = (e / N2) % N2, zl = e % N2;
          const int o = (int)(pr.r.key[kid[k0 + s]] & 7u);
          const int tx = 2 + (o & 1), ty = 2 + ((o >> 1) & 1), tz = 2 + ((o >> 2) & 1);
          const int y = yl + NG * (ty - 1), z = zl + NG * (tz - 1);
          const float *rr = rho + ((int64_t)z * B + y) * BP;
          float2 c = X[z * B + y];
          for (int x = NG * (tx - 1); x < NG * (tx + 2); ++x) {
            c.x = fmaf(-rr[x], tw[x].x, c.x);
            c.y = fmaf(-rr[x], tw[x].y, c.y);
          }
          Xn[s * N2 * N2 + yl * N2 + zl] = c;
        }
        __syncthreads();
        // direct (y, z) convolution: thread (child s, y', ys)
        if (tid < nk * NG * B) {
          const int s = tid / (NG * B), yp = (tid / B) % NG, ys = tid % B;
          const int o = (int)(pr.r.key[kid[k0 + s]] & 7u);
          const int ty = 2 + ((o >> 1) & 1), tz = 2 + ((o >> 2) & 1);
          int dy = NG * ty + yp - ys;
          dy = dy < 0 ? -dy : dy;
          const int ybase = NG * (ty - 1);
          const bool ynear = ys >= ybase && ys < ybase + N2;
          float2 *out = part + ((int64_t)(s * NG + yp) * B + ys) * NG;
          if (tz == 2) conv_row<NG, 2>(X, Xn + s * N2 * N2, ys, ynear, ybase, Kk + dy * R, out);
          else conv_row<NG, 3>(X, Xn + s * N2 * N2, ys, ynear, ybase, Kk + dy * R, out);
        }
        __syncthreads();
        // reduce over ys and accumulate the inverse transform along x
        if (owner && ok >= k0 && ok < k0 + nk) {
          const int s = ok - k0;
          float2 Y = make_float2(0.f, 0.f);
          for (int ys = 0; ys < B; ++ys) {
            const float2 v = part[((int64_t)(s * NG + oy) * B + ys) * NG + oz];
            Y.x += v.x;
            Y.y += v.y;
          }
#pragma unroll
          for (int q = 0; q < NG; ++q) {
            float sn, cs;
            sincospif(2.f * (float)((kx * (NG * otx + q)) % P) / (float)P, &sn, &cs);
            phi[q] = fmaf(wk, Y.x * cs - Y.y * sn, phi[q]);
          }
        }
      }
    }
    if (owner) {
      const int t = kid[8 + ok];
#pragma unroll
      for (int q = 0; q < NG; ++q) pr.r.out[(int64_t)t * M3 + q + NG * (oy + NG * oz)] = phi[q];
      if (oy == 0 && oz == 0) {
        const int o = (int)(pr.r.key[kid[ok]] & 7u);
        const int tx = 2 + (o & 1), ty = 2 + ((o >> 1) & 1), tz = 2 + ((o >> 2) & 1);
        float s = 0.f;
        for (int j = 0; j < 216; ++j) {
          const int bx = j % 6, by = (j / 6) % 6, bz = j / 36;
          if (max(abs(bx - tx), max(abs(by - ty), abs(bz - tz))) >= 2) s += boxsum[j];
        }
        pr.r.outc[t] = -pr.r.gmean[lev] * s;
      }
    }
    __syncthreads();
  }
}
}  // namespace xd

// ===========================================================================
// Generic path, any Ng in 1..8: the same convolution done as separable
// discrete Fourier sums per line with the same circular placement, one target
// per block at a time, intermediate spectra in per-block global scratch. The
// inverse transforms are read at the target's nodes widened by `ext` on each
// side (Sec. 2.5: ext = 1 with HPM_FLAG_EXTENDED_GRIDLET; those nodes are
// within P/2 = 4 Ng grid points of every zone source, so the periodic images
// do not reach them): positions -ext .. Ng - 1 + ext around the target's node 0.
// ===========================================================================
namespace gen {
constexpr int kThreads = 256;

struct Params {
  TreeRefs r;
  Levels lt;
  int ng;
  int ext;             // widening of the target gridlet, 0 or 1
  float2 *scratch;
  int64_t scratch_per_block;
};

__global__ void __launch_bounds__(kThreads) k_m2l_generic(const __grid_constant__ Params pr) {
  __shared__ float2 tw[64];
  __shared__ int blk[216];
  const int ng = pr.ng, P = 8 * ng, B = 6 * ng, H = P / 2 + 1, m3 = ng * ng * ng;
  const int ext = pr.ext, ne = ng + 2 * ext, me = ne * ne * ne;  // target nodes per axis / in all
  for (int e = threadIdx.x; e < P; e += blockDim.x) {
    double s, c;
    sincospi(2.0 * e / P, &s, &c);
    tw[e] = make_float2((float)c, (float)s);  // e^{+2 pi i e/P}
  }
  float2 *X1 = pr.scratch + pr.scratch_per_block * blockIdx.x;  // [kx][z][y]   H*B*B
  float2 *X2 = X1 + (int64_t)H * B * B;                          // [kx][ky][z]  H*P*B
  float2 *X4 = X2 + (int64_t)H * P * B;                          // [kx][ky][z'] H*P*ne
  float2 *X5 = X4 + (int64_t)H * P * ne;                         // [kx][y'][z'] H*ne*ne
  __syncthreads();
  for (int64_t t = blockIdx.x; t < pr.r.ntgt; t += gridDim.x) {
    const int box = pr.r.tgt_box[t];
    const int oc = (int)(pr.r.key[box] & 7u);
    const int tx = 2 + (oc & 1), ty = 2 + ((oc >> 1) & 1), tz = 2 + ((oc >> 2) & 1);
    const int n0[3] = {ng * tx, ng * ty, ng * tz};
    const int lev = level_of(pr.lt, box);
    const float *ghat = pr.r.ghat + pr.r.ghat_stride * lev;
    fill_block(pr.r, box, tx, ty, tz, blk);
    __syncthreads();
    // x: X1[kx][z][y] = sum_x rho(x,y,z) e^{-2 pi i kx ((x - n0x) mod P)/P}
    for (int64_t i = threadIdx.x; i < (int64_t)H * B * B; i += blockDim.x) {
      const int y = (int)(i % B), z = (int)((i / B) % B), kx = (int)(i / ((int64_t)B * B));
      float2 s = make_float2(0.f, 0.f);
      for (int x = 0; x < B; ++x) {
        const int row = blk[x / ng + 6 * (y / ng) + 36 * (z / ng)];
        if (row < 0) continue;
        const float v = pr.r.grid[(int64_t)row * m3 + (x % ng) + ng * ((y % ng) + ng * (z % ng))];
        const int e = (kx * ((x - n0[0] + P) % P)) % P;
        s.x += v * tw[e].x;
        s.y -= v * tw[e].y;
      }
      X1[i] = s;
    }
    __syncthreads();
    // y: X2[kx][ky][z] = sum_y X1[kx][z][y] e^{-2 pi i ky ((y - n0y) mod P)/P}
    for (int64_t i = threadIdx.x; i < (int64_t)H * P * B; i += blockDim.x) {
      const int z = (int)(i % B), ky = (int)((i / B) % P), kx = (int)(i / ((int64_t)B * P));
      float2 s = make_float2(0.f, 0.f);
      for (int y = 0; y < B; ++y) {
        const float2 v = X1[((int64_t)kx * B + z) * B + y];
        const float2 c = tw[(ky * ((y - n0[1] + P) % P)) % P];
        s.x += v.x * c.x + v.y * c.y;
        s.y += v.y * c.x - v.x * c.y;
      }
      X2[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      float sum = 0.f;
      for (int z = 0; z < B; ++z) sum += X2[z].x;  // kx = ky = 0
      pr.r.outc[t] = -pr.r.gmean[lev] * sum;
    }
    // z, Green product, inverse z to z' = -ext .. ng - 1 + ext
    for (int64_t i = threadIdx.x; i < (int64_t)H * P; i += blockDim.x) {
      const int ky = (int)(i % P), kx = (int)(i / P);
      float2 acc[kMaxNg];
      for (int q = 0; q < ne; ++q) acc[q] = make_float2(0.f, 0.f);
      const int kyr = ky <= P / 2 ? ky : P - ky;
      for (int kz = 0; kz < P; ++kz) {
        float2 s = make_float2(0.f, 0.f);
        for (int z = 0; z < B; ++z) {
          const float2 v = X2[((int64_t)kx * P + ky) * B + z];
          const float2 c = tw[(kz * ((z - n0[2] + P) % P)) % P];
          s.x += v.x * c.x + v.y * c.y;
          s.y += v.y * c.x - v.x * c.y;
        }
        const int kzr = kz <= P / 2 ? kz : P - kz;
        const float g = ghat[kx + H * (kyr + H * kzr)];
        s.x *= g;
        s.y *= g;
        for (int q = 0; q < ne; ++q) {
          const float2 c = tw[(kz * (q - ext + P)) % P];
          acc[q].x += s.x * c.x - s.y * c.y;
          acc[q].y += s.x * c.y + s.y * c.x;
        }
      }
      for (int q = 0; q < ne; ++q) X4[i * ne + q] = acc[q];
    }
    __syncthreads();
    // inverse y to y' = -ext .. ng - 1 + ext
    for (int64_t i = threadIdx.x; i < (int64_t)H * ne * ne; i += blockDim.x) {
      const int zq = (int)(i % ne), yq = (int)((i / ne) % ne), kx = (int)(i / ((int64_t)ne * ne));
      float2 s = make_float2(0.f, 0.f);
      for (int ky = 0; ky < P; ++ky) {
        const float2 v = X4[((int64_t)kx * P + ky) * ne + zq];
        const float2 c = tw[(ky * (yq - ext + P)) % P];
        s.x += v.x * c.x - v.y * c.y;
        s.y += v.x * c.y + v.y * c.x;
      }
      X5[i] = s;
    }
    __syncthreads();
    // inverse x (complex to real) to x' = -ext .. ng - 1 + ext
    for (int p = threadIdx.x; p < me; p += blockDim.x) {
      const int xq = p % ne, yq = (p / ne) % ne, zq = p / (ne * ne);
      float s = 0.f;
      for (int kx = 0; kx < H; ++kx) {
        const float2 v = X5[((int64_t)kx * ne + yq) * ne + zq];
        const float2 c = tw[(kx * (xq - ext + P)) % P];
        const float re = v.x * c.x - v.y * c.y;
        s += (kx == 0 || 2 * kx == P) ? re : 2.f * re;
      }
      pr.r.out[t * me + p] = s;
    }
    __syncthreads();
  }
}
}  // namespace gen


template <int NG>
hpm_status launch_xd(const xd::Params &p, int64_t grid, cudaStream_t st) {
  constexpr size_t smem = xd::Geo<NG>::kSmem;
  static DeviceCache attr_cache;
  int done = 0;
  HPM_TRY(device_cached(attr_cache, [](int *v) -> hpm_status {
    HPM_CUDA(cudaFuncSetAttribute(xd::k_m2l_xdft<NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    *v = 1;
    return HPM_OK;
  }, &done));
  xd::k_m2l_xdft<NG><<<(unsigned)grid, xd::Launch<NG>::threads, smem, st>>>(p);
  return HPM_OK;
}

}  // namespace

// Streaming multiprocessors of the current device (cached per device; 1 if
// the query fails).
int sm_count() {
  static DeviceCache cache;
  int n = 1;
  if (device_cached(cache, [](int *v) -> hpm_status {
        int dev = 0;
        HPM_CUDA(cudaGetDevice(&dev));
        HPM_CUDA(cudaDeviceGetAttribute(v, cudaDevAttrMultiProcessorCount, dev));
        if (*v <= 0) *v = 1;
        return HPM_OK;
      }, &n) != HPM_OK)
    return 1;
  return n;
}

hpm_status launch_m2l(hpm_plan_s *pl, cudaStream_t st, int64_t *launches) {
  TreeRefs r{};
  r.grid = pl->s.grid.as<float>();
  r.out = pl->s.m2l_raw.as<float>();
  r.outc = pl->s.m2lc.as<float>();
  r.gmean = pl->gmean.as<float>();
  r.tgt_box = pl->t.tgt_box.as<int>();
  r.parent = pl->t.box_parent.as<int>();
  r.nb = pl->t.box_nb.as<int>();
  r.child = pl->t.box_child.as<int>();
  r.key = pl->t.box_key.as<uint64_t>();
  r.ghat = pl->ghat.as<float>();
  r.ghat_stride = pl->ghat_level_stride;
  r.off2 = pl->lvl_off[2];
  r.ntgt = pl->ntgt;
  Levels lt{};
  lt.nlev = pl->max_depth + 1;
  for (int l = 0; l <= pl->max_depth + 1; ++l) lt.off[l] = pl->lvl_off[l];
  if (use_tc_m2l(pl)) return launch_m2l_tc(pl, st, launches);
  const int nsm = sm_count();
  const bool extended = (pl->opts.flags & HPM_FLAG_EXTENDED_GRIDLET) != 0;  // any-order kernel only
  if (pl->ng == 4 && !extended && !(pl->opts.flags & (HPM_FLAG_GENERIC_M2L | HPM_FLAG_XTRANSFORM_M2L))) {
    f4::Params p{};
    for (int e = 0; e < f4::kP; ++e) {
      const double a = -2.0 * M_PI * e / f4::kP;
      p.w[e] = make_float2((float)cos(a), (float)sin(a));
    }
    p.r = r;
    p.lt = lt;
    p.kz = pl->kz_green.as<float>();
    p.kz_stride = pl->kz_green_stride;
    p.tblk = pl->t.tgt_blk.as<int>();
    p.tinfo = pl->t.tgt_info.as<int>();
    static DeviceCache attr_cache;
    int done = 0;
    HPM_TRY(device_cached(attr_cache, [](int *v) -> hpm_status {
      HPM_CUDA(cudaFuncSetAttribute(f4::k_m2l4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f4::kSmem));
      *v = 1;
      return HPM_OK;
    }, &done));
    const int per_sm = pl->tuning.m2l_ctas_per_sm == 1 ? 1 : 2;  // 2 fit (111 KB each)
    const int64_t grid = std::min<int64_t>(pl->ntgt, (int64_t)per_sm * nsm);
    f4::k_m2l4<<<(unsigned)grid, f4::kThreads, f4::kSmem, st>>>(p);
    HPM_LAUNCHED(launches);
    return HPM_OK;
  }
  const bool xd_order = pl->ng == 2 || pl->ng == 3 || pl->ng == 5 || pl->ng == 6 ||
                        (pl->ng == 4 && (pl->opts.flags & HPM_FLAG_XTRANSFORM_M2L));
  if (!(pl->opts.flags & HPM_FLAG_GENERIC_M2L) && xd_order && !extended) {
    xd::Params p{};
    p.r = r;
    p.lt = lt;
    p.par_box = pl->t.par_box.as<int>();
    p.box_tgt = pl->t.box_tgt.as<int>();
    p.npar = pl->npar;
    p.kxg = pl->kx_green.as<float>();
    p.kx_stride = pl->kx_green_stride;
    // persistent CTAs per SM: two fit up to Ng = 4, one above; the tuner may take fewer
    const int per_sm = std::min(pl->ng <= 4 ? 2 : 1, pl->tuning.m2l_ctas_per_sm > 0 ? pl->tuning.m2l_ctas_per_sm : 2);
    const int64_t grid = std::min<int64_t>(pl->npar, (int64_t)nsm * per_sm);
    if (grid <= 0) return HPM_OK;
    switch (pl->ng) {
      case 2: HPM_TRY(launch_xd<2>(p, grid, st)); break;
      case 3: HPM_TRY(launch_xd<3>(p, grid, st)); break;
      case 4: HPM_TRY(launch_xd<4>(p, grid, st)); break;
      case 5: HPM_TRY(launch_xd<5>(p, grid, st)); break;
      default: HPM_TRY(launch_xd<6>(p, grid, st)); break;
    }
    HPM_LAUNCHED(launches);
    return HPM_OK;
  }
  gen::Params p{};
  p.r = r;
  p.lt = lt;
  p.ng = pl->ng;
  p.ext = extended ? 1 : 0;
  const int P = 8 * pl->ng, B = 6 * pl->ng, H = P / 2 + 1, ne = pl->ng + 2 * p.ext;
  p.scratch_per_block = (int64_t)H * B * B + (int64_t)H * P * B + (int64_t)H * P * ne + (int64_t)H * ne * ne;
  const int64_t grid = std::min<int64_t>(pl->ntgt, (int64_t)nsm);
  HPM_TRY(pl->s.m2l_scratch.ensure(sizeof(float2) * p.scratch_per_block * grid, st));
  p.scratch = pl->s.m2l_scratch.as<float2>();
  gen::k_m2l_generic<<<(unsigned)grid, gen::kThreads, 0, st>>>(p);
  HPM_LAUNCHED(launches);
  return HPM_OK;
}

}  // namespace hpm
