// The Green function, evaluated on the host in FP64 (Sec. 4: the method only
// convolves with g, so any radial kernel serves; Sec. 2.1, Eq. gf: it is
// tabulated exactly on the gridlet lattice before any timing).
//
//   lattice tables  G_l[n] = g(h_l sqrt(n)) for the integers n = |d|^2 of every
//                   lattice offset d a level-l convolution meets (grid spacing
//                   h_l = S / (2^l Ng)); G_l[0] takes the value at unit offset
//                   (the softened zero of Sec. 2.1, which never reaches a
//                   target value). Every far-field table of the plan (Green
//                   transforms, the dense tensor-core matrices) is built on the
//                   device from these FP64 values.
//   near table      (user kernels only) piecewise cubics of g and of the force
//                   factor F = -g'(r) / r_u in the FP32 bits of r_u^2 (r_u the
//                   distance in units of the domain side): 32 segments per
//                   octave of r_u^2 over [2^-64, 4), each a cubic in the
//                   segment's mantissa fraction through g and F at the four
//                   Chebyshev-Lobatto points of the segment. Below 2^-64 the
//                   values at 2^-64 are used (documented in include/hpm.h).
#include <cmath>
#include <vector>

#include "hpm_internal.cuh"

namespace hpm {

double green_g(const hpm_green &g, double r) {
  switch (g.kind) {
    case HPM_GREEN_NEWTON:
      return 1.0 / r;
    case HPM_GREEN_YUKAWA: {
      const double s = std::sqrt(r * r + g.eps * g.eps);
      return std::exp(-s / g.lambda) / s;
    }
    case HPM_GREEN_USER:
      return g.user_g(r, g.ctx);
    default: {
      return 1.0 / std::sqrt(r * r + g.eps * g.eps);
    }
  }
}

// -g'(r): central differences at steps h and h/2 combined by Richardson
// extrapolation (fourth order); h = r / 512 keeps the truncation near 1e-11
// and the rounding near 1e-13 relative for kernels smooth on that scale.
static double green_minus_dg(const hpm_green &g, double r) {
  const double h = r / 512.0;
  const double d1 = (green_g(g, r + h) - green_g(g, r - h)) / (2.0 * h);
  const double d2 = (green_g(g, r + 0.5 * h) - green_g(g, r - 0.5 * h)) / h;
  return -(4.0 * d2 - d1) / 3.0;
}

int64_t lattice_nmax(int ng) {
  // FFT-form tables: offsets up to P/2 = 4 Ng per axis; the dense product:
  // offsets up to 6 Ng - 1 per axis inside a parent's 6^3 block
  const int64_t a = 3 * (int64_t)(4 * ng) * (4 * ng), b = 3 * (int64_t)(6 * ng - 1) * (6 * ng - 1);
  return a > b ? a : b;
}

hpm_status build_lattice(hpm_plan_s *pl, cudaStream_t st) {
  const int D = pl->max_depth;
  const int64_t nn = lattice_nmax(pl->ng) + 1;
  pl->glat_stride = nn;
  pl->glat_host.assign((size_t)nn * (D + 1), 0.0);
  for (int l = 2; l <= D; ++l) {
    const double h = pl->dom.side / (double)(1u << l) / (double)pl->ng;
    double *row = pl->glat_host.data() + (size_t)nn * l;
    for (int64_t n = 1; n < nn; ++n) {
      row[n] = green_g(pl->green, h * std::sqrt((double)n));
      if (!std::isfinite(row[n])) return HPM_ERR_INVALID_ARG;
    }
    row[0] = row[1];  // g(0) := g(unit offset), Sec. 2.1
  }
  HPM_TRY(pl->glat.ensure(sizeof(double) * pl->glat_host.size(), st));
  HPM_CUDA(cudaMemcpyAsync(pl->glat.p, pl->glat_host.data(), sizeof(double) * pl->glat_host.size(),
                           cudaMemcpyHostToDevice, st));
  return HPM_OK;
}

hpm_status build_near_table(hpm_plan_s *pl, cudaStream_t st) {
  if (pl->green.kind != HPM_GREEN_USER) return HPM_OK;
  constexpr int nseg = kNearTabOctaves * kNearTabSeg;
  std::vector<float> tab((size_t)nseg * 8);
  const double S = pl->dom.side;
  // Chebyshev-Lobatto points of [0, 1] and the inverse of their Vandermonde
  // matrix (monomials 1, t, t^2, t^3)
  const double tn[4] = {0.0, 0.25, 0.75, 1.0};
  double V[4][4], Vi[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      V[i][j] = std::pow(tn[i], j);
      Vi[i][j] = i == j ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {  // Gauss-Jordan with partial pivoting
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::fabs(V[r][c]) > std::fabs(V[p][c])) p = r;
    for (int k = 0; k < 4; ++k) {
      std::swap(V[c][k], V[p][k]);
      std::swap(Vi[c][k], Vi[p][k]);
    }
    const double d = V[c][c];
    for (int k = 0; k < 4; ++k) {
      V[c][k] /= d;
      Vi[c][k] /= d;
    }
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        const double f = V[r][c];
        for (int k = 0; k < 4; ++k) {
          V[r][k] -= f * V[c][k];
          Vi[r][k] -= f * Vi[c][k];
        }
      }
  }
  for (int s = 0; s < nseg; ++s) {
    const int e = kNearTabE0 + s / kNearTabSeg, m = s % kNearTabSeg;
    double gv[4], fv[4];
    for (int i = 0; i < 4; ++i) {
      const double r2 = std::ldexp(1.0 + (m + tn[i]) / kNearTabSeg, e);  // r_u^2
      const double ru = std::sqrt(r2);
      gv[i] = green_g(pl->green, S * ru);
      fv[i] = green_minus_dg(pl->green, S * ru) / ru;  // -g'(r) / r_u
      if (!std::isfinite(gv[i]) || !std::isfinite(fv[i])) return HPM_ERR_INVALID_ARG;
    }
    for (int j = 0; j < 4; ++j) {
      double cg = 0.0, cf = 0.0;
      for (int i = 0; i < 4; ++i) {
        cg += Vi[j][i] * gv[i];
        cf += Vi[j][i] * fv[i];
      }
      tab[(size_t)s * 8 + j] = (float)cg;
      tab[(size_t)s * 8 + 4 + j] = (float)cf;
    }
  }
  HPM_TRY(pl->near_tab.ensure(sizeof(float) * tab.size(), st));
  HPM_CUDA(cudaMemcpyAsync(pl->near_tab.p, tab.data(), sizeof(float) * tab.size(), cudaMemcpyHostToDevice, st));
  // the copy reads a host vector that goes out of scope: wait for it
  HPM_CUDA(cudaStreamSynchronize(st));
  return HPM_OK;
}

}  // namespace hpm
