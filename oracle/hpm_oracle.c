/*
 * FP64 CPU oracle for the Hierarchical Particle-Mesh FMM (Gnedin 2019,
 * "Hierarchical Particle-Mesh: an FFT-accelerated Fast Multipole Method").
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this library. The GPU solver
 * never calls, links or includes anything from here, and this file shares no
 * code, header, table or constant generator with the CUDA kernels.
 *
 * Everything is FP64 and written as the plain definition of each step:
 *   - gridlet effective masses of a box straight from its particles with the
 *     Lagrange weights (Sec. 2.2, Eq. mp, since sum_n B_pn t^n is the
 *     Lagrange basis polynomial of node p), and in the paper's own form
 *     (Cartesian multipoles Q_n, Eq. cm, then M = B (n!/L^n) Q, Eq. mp);
 *   - the child-to-parent matrices T^C of Sec. 2.3 from the paper's double
 *     sum over multi-indices;
 *   - the source-to-target transformation as the direct double sum over the
 *     interaction-zone effective masses, and as the paper's zero-padded
 *     (8 Ng)^3 periodic convolution with the exact Green function (Sec. 2.1,
 *     Eq. gf) done with a plain mixed-radix complex FFT written here;
 *   - the far field at a particle as the sum over the target cell and its
 *     ancestors of the interpolating polynomial of Eqs. c2pmat/phix and its
 *     analytic gradient;
 *   - near-zone and all-pairs direct summation.
 *
 * Kernel: any radial Green function g (Sec. 4: the method only convolves
 * with it), given as an or_kernel: Plummer 1/sqrt(r^2 + eps^2), Newton 1/r,
 * Yukawa exp(-s/lambda)/s with s = sqrt(r^2 + eps^2), or a user function
 * g(r, ctx) with an optional derivative. Potential phi_i = -sum_j m_j g(r_ij),
 * acceleration a = -grad phi (G = 1, the 1/(4 pi) of Eq. gf dropped).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------------------
 * The Green function. kind: 0 Plummer, 1 Newton, 2 Yukawa, 3 user.
 * A user kernel gives g(r, ctx) and, optionally, dg(r, ctx) = g'(r); without
 * dg the derivative is the sixth-order central difference at step r/1000.
 * User kernels are evaluated at r >= rmin (closer pairs take the values at
 * rmin, the library's documented cut-off side * 2^-32).
 * ------------------------------------------------------------------------- */
typedef struct {
  int kind;
  double eps, lambda, rmin;
  double (*user_g)(double r, void *ctx);
  double (*user_dg)(double r, void *ctx);
  void *ctx;
} or_kernel;

static double or_g(const or_kernel *k, double r) {
  switch (k->kind) {
    case 1: return 1.0 / r;
    case 2: {
      const double s = sqrt(r * r + k->eps * k->eps);
      return exp(-s / k->lambda) / s;
    }
    case 3: return k->user_g(r < k->rmin ? k->rmin : r, k->ctx);
    default: return 1.0 / sqrt(r * r + k->eps * k->eps);
  }
}

/* F(r) = -g'(r)/r: the pair term of the acceleration is a_i += m_j F (x_j - x_i). */
static double or_force_factor(const or_kernel *k, double r) {
  switch (k->kind) {
    case 1: return 1.0 / (r * r * r);
    case 2: {
      const double s = sqrt(r * r + k->eps * k->eps);
      return exp(-s / k->lambda) * (1.0 + s / k->lambda) / (s * s * s);
    }
    case 3: {
      const double x = r < k->rmin ? k->rmin : r;
      double d;
      if (k->user_dg) {
        d = k->user_dg(x, k->ctx);
      } else {
        const double h = x / 1000.0;
        d = (-k->user_g(x - 3 * h, k->ctx) + 9 * k->user_g(x - 2 * h, k->ctx) - 45 * k->user_g(x - h, k->ctx) +
             45 * k->user_g(x + h, k->ctx) - 9 * k->user_g(x + 2 * h, k->ctx) + k->user_g(x + 3 * h, k->ctx)) /
            (60.0 * h);
      }
      return -d / x;
    }
    default: {
      const double r2 = r * r + k->eps * k->eps;
      return 1.0 / (r2 * sqrt(r2));
    }
  }
}

/* Exported for the pins: g(r) and F(r) at n distances. */
void or_kernel_eval(const or_kernel *k, int64_t n, const double *r, double *g, double *f) {
  for (int64_t i = 0; i < n; ++i) {
    if (g) g[i] = or_g(k, r[i]);
    if (f) f[i] = or_force_factor(k, r[i]);
  }
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Gridlet node coordinate in box units, Sec. 2.2: x_j = (j + 1/2)/Ng - 1/2. */
static double node_x(int j, int ng) { return (j + 0.5) / ng - 0.5; }

/* Lagrange basis ell_j(t) on the Ng gridlet nodes, and its derivative. */
void or_lagrange(int ng, double t, double *w, double *dw) {
  for (int j = 0; j < ng; ++j) {
    double xj = node_x(j, ng), v = 1.0;
    for (int k = 0; k < ng; ++k)
      if (k != j) v *= (t - node_x(k, ng)) / (xj - node_x(k, ng));
    w[j] = v;
    if (dw) {
      double d = 0.0;
      for (int m = 0; m < ng; ++m) {
        if (m == j) continue;
        double term = 1.0 / (xj - node_x(m, ng));
        for (int k = 0; k < ng; ++k)
          if (k != j && k != m) term *= (t - node_x(k, ng)) / (xj - node_x(k, ng));
        d += term;
      }
      dw[j] = d;
    }
  }
}

/* Lagrange basis on the extended target gridlet of Sec. 2.5: the Ng nodes of
 * the cell widened by `ext` nodes of the same spacing on each side, nodes
 * x_j = (j + 1/2)/Ng - 1/2 for j = -ext .. Ng - 1 + ext (ext = 0: the gridlet
 * itself). w and dw get Ng + 2 ext values. */
void or_lagrange_ext(int ng, int ext, double t, double *w, double *dw) {
  const int ne = ng + 2 * ext;
  for (int j = 0; j < ne; ++j) {
    const double xj = node_x(j - ext, ng);
    double v = 1.0;
    for (int k = 0; k < ne; ++k)
      if (k != j) v *= (t - node_x(k - ext, ng)) / (xj - node_x(k - ext, ng));
    w[j] = v;
    if (dw) {
      double d = 0.0;
      for (int m = 0; m < ne; ++m) {
        if (m == j) continue;
        double term = 1.0 / (xj - node_x(m - ext, ng));
        for (int k = 0; k < ne; ++k)
          if (k != j && k != m) term *= (t - node_x(k - ext, ng)) / (xj - node_x(k - ext, ng));
        d += term;
      }
      dw[j] = d;
    }
  }
}

/* ---------------------------------------------------------------------------
 * P2G, Lagrange form. For box b with centre c and side L:
 *   M_{b,p} = sum_{i in b} m_i prod_d ell_{p_d}(xi_{i,d}),  xi = (x_i - c)/L.
 * Particles of box b are pos[begin[b] .. end[b]) (pos in the sorted order).
 * Output row b holds Ng^3 values, node p = i + Ng j + Ng^2 k.
 * ------------------------------------------------------------------------- */
void or_p2g(int ng, int64_t nbox, const int64_t *begin, const int64_t *end,
            const double *center, const double *side, const double *pos,
            const double *mass, double *out) {
  const int m3 = ng * ng * ng;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nbox; ++b) {
    double wx[16], wy[16], wz[16];
    double *o = out + b * m3;
    for (int p = 0; p < m3; ++p) o[p] = 0.0;
    for (int64_t i = begin[b]; i < end[b]; ++i) {
      or_lagrange(ng, (pos[3 * i + 0] - center[3 * b + 0]) / side[b], wx, NULL);
      or_lagrange(ng, (pos[3 * i + 1] - center[3 * b + 1]) / side[b], wy, NULL);
      or_lagrange(ng, (pos[3 * i + 2] - center[3 * b + 2]) / side[b], wz, NULL);
      for (int k = 0; k < ng; ++k)
        for (int j = 0; j < ng; ++j)
          for (int ii = 0; ii < ng; ++ii)
            o[ii + ng * (j + ng * k)] += mass[i] * wx[ii] * wy[j] * wz[k];
    }
  }
}

/* ---------------------------------------------------------------------------
 * The paper's own form of P2G (Sec. 2.2).
 * Multi-index n = (nx, ny, nz), raveled n = nx + Ng ny + Ng^2 nz.
 * ------------------------------------------------------------------------- */
static double factorial(int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; }

/* Vandermonde matrix of Eq. Anp: A[n][p] = x_p^n (row n, column p). */
void or_vandermonde(int ng, double *A) {
  const int m3 = ng * ng * ng;
  for (int n = 0; n < m3; ++n) {
    int nx = n % ng, ny = (n / ng) % ng, nz = n / (ng * ng);
    for (int p = 0; p < m3; ++p) {
      int px = p % ng, py = (p / ng) % ng, pz = p / (ng * ng);
      A[n * m3 + p] = pow(node_x(px, ng), nx) * pow(node_x(py, ng), ny) * pow(node_x(pz, ng), nz);
    }
  }
}

/* Inverse of an n x n matrix by Gauss-Jordan elimination with partial pivoting.
 * Returns 0 on success, -1 for a singular matrix. */
int or_invert(int n, const double *A, double *Ainv) {
  double *a = (double *)malloc(sizeof(double) * n * n);
  memcpy(a, A, sizeof(double) * n * n);
  for (int i = 0; i < n * n; ++i) Ainv[i] = 0.0;
  for (int i = 0; i < n; ++i) Ainv[i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(a[r * n + c]) > fabs(a[piv * n + c])) piv = r;
    if (a[piv * n + c] == 0.0) { free(a); return -1; }
    if (piv != c)
      for (int k = 0; k < n; ++k) {
        double t = a[c * n + k]; a[c * n + k] = a[piv * n + k]; a[piv * n + k] = t;
        t = Ainv[c * n + k]; Ainv[c * n + k] = Ainv[piv * n + k]; Ainv[piv * n + k] = t;
      }
    double d = a[c * n + c];
    for (int k = 0; k < n; ++k) { a[c * n + k] /= d; Ainv[c * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[c * n + k]; Ainv[r * n + k] -= f * Ainv[c * n + k]; }
    }
  }
  free(a);
  return 0;
}

/* Cartesian multipoles of Eq. cm for each box, about the box centre:
 *   Q_n = (1/n!) sum_i m_i r_i^n,  r = x - c (physical units). */
void or_moments(int ng, int64_t nbox, const int64_t *begin, const int64_t *end,
                const double *center, const double *pos, const double *mass, double *Q) {
  const int m3 = ng * ng * ng;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t b = 0; b < nbox; ++b) {
    double *q = Q + b * m3;
    for (int n = 0; n < m3; ++n) q[n] = 0.0;
    for (int64_t i = begin[b]; i < end[b]; ++i) {
      double r[3];
      for (int d = 0; d < 3; ++d) r[d] = pos[3 * i + d] - center[3 * b + d];
      for (int n = 0; n < m3; ++n) {
        int nx = n % ng, ny = (n / ng) % ng, nz = n / (ng * ng);
        q[n] += mass[i] * pow(r[0], nx) * pow(r[1], ny) * pow(r[2], nz);
      }
    }
    for (int n = 0; n < m3; ++n) {
      int nx = n % ng, ny = (n / ng) % ng, nz = n / (ng * ng);
      q[n] /= factorial(nx) * factorial(ny) * factorial(nz);
    }
  }
}

/* Eq. mp: M_p = sum_n B[p][n] (n!/L^n) Q_n, for boxes of side L[b]. */
void or_p2g_paper(int ng, int64_t nbox, const double *Q, const double *side,
                  const double *B, double *out) {
  const int m3 = ng * ng * ng;
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nbox; ++b) {
    for (int p = 0; p < m3; ++p) {
      double s = 0.0;
      for (int n = 0; n < m3; ++n) {
        int nx = n % ng, ny = (n / ng) % ng, nz = n / (ng * ng);
        double f = factorial(nx) * factorial(ny) * factorial(nz) / pow(side[b], nx + ny + nz);
        s += B[p * m3 + n] * f * Q[b * m3 + n];
      }
      out[b * m3 + p] = s;
    }
  }
}

/* Child-to-parent matrix of Sec. 2.3:
 *   T^C_pq = sum_n sum_{m <= n} B_pn n!/(m!(n-m)!) (a^C)^(n-m) / 2^|n| A_mq,
 * with a^C the child centre in units where the parent spans [-1, 1]:
 * a = (+-1/2, +-1/2, +-1/2), child index C = bx + 2 by + 4 bz, bit set = '+'.
 * (The two printed lines of the derivation swap m and n-m; by the binomial
 * symmetry both orderings give the same matrix, used here as printed last.) */
void or_t_paper(int ng, const double *A, const double *B, int child, double *T) {
  const int m3 = ng * ng * ng;
  double a[3];
  for (int d = 0; d < 3; ++d) a[d] = ((child >> d) & 1) ? 0.5 : -0.5;
  /* C_nm = n!/(m!(n-m)!) a^(n-m) / 2^|n| for m <= n componentwise, else 0 */
  double *Cnm = (double *)calloc((size_t)m3 * m3, sizeof(double));
  for (int n = 0; n < m3; ++n) {
    int nn[3] = {n % ng, (n / ng) % ng, n / (ng * ng)};
    for (int m = 0; m < m3; ++m) {
      int mm[3] = {m % ng, (m / ng) % ng, m / (ng * ng)};
      double v = 1.0;
      for (int d = 0; d < 3 && v != 0.0; ++d) {
        if (mm[d] > nn[d]) { v = 0.0; break; }
        v *= factorial(nn[d]) / (factorial(mm[d]) * factorial(nn[d] - mm[d])) *
             pow(a[d], nn[d] - mm[d]) / pow(2.0, nn[d]);
      }
      Cnm[n * m3 + m] = v;
    }
  }
  for (int p = 0; p < m3; ++p)
    for (int q = 0; q < m3; ++q) {
      double s = 0.0;
      for (int n = 0; n < m3; ++n) {
        double bpn = B[p * m3 + n];
        if (bpn == 0.0) continue;
        double inner = 0.0;
        for (int m = 0; m < m3; ++m) inner += Cnm[n * m3 + m] * A[m * m3 + q];
        s += bpn * inner;
      }
      T[p * m3 + q] = s;
    }
  free(Cnm);
}

/* ---------------------------------------------------------------------------
 * Source-to-target transformation, direct double sum (plain definition):
 *   Phi_{t,p} = - sum_{b in IZ(t)} sum_q M_{b,q} g(|y_{t,p} - y_{b,q}|),
 * node positions y = c + L x_p. Sources of target t are rows
 * sidx[soff[t] .. soff[t+1]) of the source tables. The target's nodes may be
 * the extended gridlet of Sec. 2.5 (ext = 1: one more node on each side,
 * (Ng + 2)^3 values per target); the sources are always Ng^3 gridlets.
 * ------------------------------------------------------------------------- */
void or_m2l_direct(int ng, int ext, const or_kernel *kern, int64_t ntgt, const double *tcenter,
                   const double *tside, const int64_t *soff, const int64_t *sidx, const double *scenter,
                   const double *sgrid, double *out) {
  const int m3 = ng * ng * ng, ne = ng + 2 * ext, me = ne * ne * ne;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t t = 0; t < ntgt; ++t) {
    const double L = tside[t];
    for (int p = 0; p < me; ++p) {
      double yp[3] = {tcenter[3 * t + 0] + L * node_x(p % ne - ext, ng),
                      tcenter[3 * t + 1] + L * node_x((p / ne) % ne - ext, ng),
                      tcenter[3 * t + 2] + L * node_x(p / (ne * ne) - ext, ng)};
      double s = 0.0;
      for (int64_t e = soff[t]; e < soff[t + 1]; ++e) {
        const int64_t b = sidx[e];
        for (int q = 0; q < m3; ++q) {
          double dx = yp[0] - (scenter[3 * b + 0] + L * node_x(q % ng, ng));
          double dy = yp[1] - (scenter[3 * b + 1] + L * node_x((q / ng) % ng, ng));
          double dz = yp[2] - (scenter[3 * b + 2] + L * node_x(q / (ng * ng), ng));
          s += sgrid[b * m3 + q] * or_g(kern, sqrt(dx * dx + dy * dy + dz * dz));
        }
      }
      out[t * me + p] = -s;
    }
  }
}

/* ---------------------------------------------------------------------------
 * Plain mixed-radix complex FFT (decimation in time, smallest prime factor
 * first). sign = -1 forward, +1 backward (unnormalised).
 * ------------------------------------------------------------------------- */
static int smallest_factor(int n) {
  for (int r = 2; r * r <= n; ++r)
    if (n % r == 0) return r;
  return n;
}

static void fft_rec(cplx *out, const cplx *in, int n, int stride, const cplx *tw, int twn,
                    cplx *work) {
  if (n == 1) { out[0] = in[0]; return; }
  const int r = smallest_factor(n), m = n / r;
  cplx *sub = work, *deeper = work + n;
  for (int j = 0; j < r; ++j) fft_rec(sub + j * m, in + j * stride, m, stride * r, tw, twn, deeper);
  const int step = twn / n;          /* W_n^e = W_twn^(e * twn / n) */
  for (int k = 0; k < m; ++k)
    for (int s = 0; s < r; ++s) {
      const int kk = k + m * s;
      cplx acc = 0.0;
      for (int j = 0; j < r; ++j) acc += tw[(int64_t)((int64_t)j * kk % n) * step] * sub[j * m + k];
      out[kk] = acc;
    }
}

/* 3-D transform of a P^3 array (x fastest), line by line along each axis. */
static void fft3d(cplx *a, int P, int sign) {
  cplx *tw = (cplx *)malloc(sizeof(cplx) * P);
  for (int k = 0; k < P; ++k) tw[k] = cexp(sign * 2.0 * M_PI * I * (double)k / (double)P);
  cplx *line = (cplx *)malloc(sizeof(cplx) * P), *res = (cplx *)malloc(sizeof(cplx) * P);
  cplx *work = (cplx *)malloc(sizeof(cplx) * 4 * P);
  const int64_t st[3] = {1, P, (int64_t)P * P};
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t s = st[ax];
    for (int64_t u = 0; u < (int64_t)P * P; ++u) {
      /* base index of line u along axis ax */
      int64_t i1 = u % P, i2 = u / P, base;
      if (ax == 0) base = i1 * P + i2 * P * P;
      else if (ax == 1) base = i1 + i2 * P * P;
      else base = i1 + i2 * P;
      for (int k = 0; k < P; ++k) line[k] = a[base + k * s];
      fft_rec(res, line, P, 1, tw, P, work);
      for (int k = 0; k < P; ++k) a[base + k * s] = res[k];
    }
  }
  free(work); free(res); free(line); free(tw);
}

/* 1-D transform, exported for the FFT pin against a direct DFT. */
void or_fft1d(const double *re_in, const double *im_in, int n, int sign, double *re_out, double *im_out) {
  cplx *tw = (cplx *)malloc(sizeof(cplx) * n), *in = (cplx *)malloc(sizeof(cplx) * n);
  cplx *out = (cplx *)malloc(sizeof(cplx) * n), *work = (cplx *)malloc(sizeof(cplx) * 4 * n);
  for (int k = 0; k < n; ++k) { tw[k] = cexp(sign * 2.0 * M_PI * I * (double)k / (double)n); in[k] = re_in[k] + I * im_in[k]; }
  fft_rec(out, in, n, 1, tw, n, work);
  for (int k = 0; k < n; ++k) { re_out[k] = creal(out[k]); im_out[k] = cimag(out[k]); }
  free(work); free(out); free(in); free(tw);
}

/* Exact Green function on the P^3 periodic grid of spacing h, Eq. gf with
 * the kernel g in place of 1/(4 pi r): G[d] = g(h |d|_p),
 * |d|_p the periodic distance per axis; G at d = 0 takes the value at unit
 * offset (Sec. 2.1). Returns its forward transform (complex, P^3). */
void or_green_hat(int P, const or_kernel *kern, double h, double *re, double *im) {
  const int64_t n3 = (int64_t)P * P * P;
  cplx *a = (cplx *)malloc(sizeof(cplx) * n3);
  for (int k = 0; k < P; ++k)
    for (int j = 0; j < P; ++j)
      for (int i = 0; i < P; ++i) {
        int di = i <= P / 2 ? i : P - i, dj = j <= P / 2 ? j : P - j, dk = k <= P / 2 ? k : P - k;
        double r2 = (double)di * di + (double)dj * dj + (double)dk * dk;
        if (r2 == 0.0) r2 = 1.0;
        a[i + (int64_t)P * (j + (int64_t)P * k)] = or_g(kern, h * sqrt(r2));
      }
  fft3d(a, P, -1);
  for (int64_t e = 0; e < n3; ++e) { re[e] = creal(a[e]); im[e] = cimag(a[e]); }
  free(a);
}

/* Source-to-target by one FFT convolution per target (Sec. 2.1). The
 * (6 Ng)^3 block covers the level-l boxes that are children of the 3^3
 * neighbourhood of the target's parent; blk[t][bx + 6 by + 36 bz] is the row
 * of that box's effective masses in grid[], or -1 where the box is empty,
 * outside the domain or in the target's near zone. The block is zero padded
 * to P^3 = (8 Ng)^3, convolved with the Green function (forward FFT, product
 * with ghat, backward FFT, 1/P^3), and the values at the target's nodes are
 * read, the (Ng + 2 ext)^3 nodes of its gridlet widened by ext on each side
 * (Sec. 2.5); tpos[t] is the target's box position in the block (2 or 3 per
 * axis). Output: Phi_{t,p} = -(G * rho)(target node p). */
void or_m2l_fft(int ng, int ext, int64_t ntgt, const int32_t *blk, const int32_t *tpos,
                const double *grid, const double *ghat_re, const double *ghat_im, double *out) {
  const int P = 8 * ng, m3 = ng * ng * ng, ne = ng + 2 * ext, me = ne * ne * ne;
  const int64_t n3 = (int64_t)P * P * P;
#pragma omp parallel
  {
    cplx *a = (cplx *)malloc(sizeof(cplx) * n3);
#pragma omp for schedule(dynamic, 1)
    for (int64_t t = 0; t < ntgt; ++t) {
      for (int64_t e = 0; e < n3; ++e) a[e] = 0.0;
      for (int bz = 0; bz < 6; ++bz)
        for (int by = 0; by < 6; ++by)
          for (int bx = 0; bx < 6; ++bx) {
            int32_t row = blk[t * 216 + bx + 6 * by + 36 * bz];
            if (row < 0) continue;
            for (int q = 0; q < m3; ++q) {
              int x = bx * ng + q % ng, y = by * ng + (q / ng) % ng, z = bz * ng + q / (ng * ng);
              a[x + (int64_t)P * (y + (int64_t)P * z)] = grid[(int64_t)row * m3 + q];
            }
          }
      fft3d(a, P, -1);
      for (int64_t e = 0; e < n3; ++e) a[e] *= ghat_re[e] + I * ghat_im[e];
      fft3d(a, P, +1);
      for (int p = 0; p < me; ++p) {
        /* periodic positions: the grid repeats every P points */
        int x = (tpos[3 * t + 0] * ng - ext + p % ne + P) % P, y = (tpos[3 * t + 1] * ng - ext + (p / ne) % ne + P) % P,
            z = (tpos[3 * t + 2] * ng - ext + p / (ne * ne) + P) % P;
        out[t * me + p] = -creal(a[x + (int64_t)P * (y + (int64_t)P * z)]) / (double)n3;
      }
    }
    free(a);
  }
}

/* ---------------------------------------------------------------------------
 * Far field at particles, plain definition of the downward pass: the sum over
 * the cells of the particle's chain (its leaf and the leaf's ancestors down to
 * level 2) of the interpolating polynomial of the cell's local gridlet,
 *   phi_i = sum_cells sum_p Phi_{c,p} prod_d ell_{p_d}(xi_d),
 *   a_i   = - sum_cells (1/L_c) sum_p Phi_{c,p} grad_xi prod_d ell_{p_d}(xi_d),
 * xi = (x_i - c)/L_c. Cells of particle i are ccell[coff[i] .. coff[i+1]).
 * The gridlets may be extended by ext nodes on each side (Sec. 2.5): the
 * interpolant is then of degree Ng - 1 + 2 ext through (Ng + 2 ext)^3 values.
 * ------------------------------------------------------------------------- */
void or_far_eval(int ng, int ext, int64_t npart, const double *pos, const int64_t *coff,
                 const int64_t *ccell, const double *ccenter, const double *cside,
                 const double *cphi, double *phi, double *acc) {
  const int ne = ng + 2 * ext, m3 = ne * ne * ne;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < npart; ++i) {
    double f = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int64_t e = coff[i]; e < coff[i + 1]; ++e) {
      const int64_t c = ccell[e];
      const double L = cside[c];
      double w[3][16], dw[3][16];
      for (int d = 0; d < 3; ++d) or_lagrange_ext(ng, ext, (pos[3 * i + d] - ccenter[3 * c + d]) / L, w[d], dw[d]);
      for (int p = 0; p < m3; ++p) {
        int px = p % ne, py = (p / ne) % ne, pz = p / (ne * ne);
        double v = cphi[c * m3 + p];
        f += v * w[0][px] * w[1][py] * w[2][pz];
        g[0] += v * dw[0][px] * w[1][py] * w[2][pz] / L;
        g[1] += v * w[0][px] * dw[1][py] * w[2][pz] / L;
        g[2] += v * w[0][px] * w[1][py] * dw[2][pz] / L;
      }
    }
    phi[i] = f;
    for (int d = 0; d < 3; ++d) acc[3 * i + d] = -g[d];
  }
}

/* The paper's form of the interpolant, Eqs. c2pmat and phix: V_n = sum_p
 * B_pn Phi_p and Phi(x) = sum_n V_n x^n, with x = (x_i - c)/L; gradient by
 * differentiating the monomials. V holds one row of Ng^3 per cell. */
void or_g2p_paper(int ng, int64_t npart, const double *pos, const int64_t *cell,
                  const double *ccenter, const double *cside, const double *V,
                  double *phi, double *acc) {
  const int m3 = ng * ng * ng;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < npart; ++i) {
    const int64_t c = cell[i];
    const double L = cside[c];
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = (pos[3 * i + d] - ccenter[3 * c + d]) / L;
    double f = 0.0, g[3] = {0.0, 0.0, 0.0};
    for (int n = 0; n < m3; ++n) {
      int nn[3] = {n % ng, (n / ng) % ng, n / (ng * ng)};
      double pw[3], dpw[3];
      for (int d = 0; d < 3; ++d) {
        pw[d] = pow(x[d], nn[d]);
        dpw[d] = nn[d] > 0 ? nn[d] * pow(x[d], nn[d] - 1) : 0.0;
      }
      double v = V[c * m3 + n];
      f += v * pw[0] * pw[1] * pw[2];
      g[0] += v * dpw[0] * pw[1] * pw[2] / L;
      g[1] += v * pw[0] * dpw[1] * pw[2] / L;
      g[2] += v * pw[0] * pw[1] * dpw[2] / L;
    }
    phi[i] += f;
    for (int d = 0; d < 3; ++d) acc[3 * i + d] -= g[d];
  }
}

/* ---------------------------------------------------------------------------
 * Near field: for target particle i (row tidx[i] of pos), sum over the
 * particle index ranges [rbeg[e], rend[e]) for e in roff[i] .. roff[i+1],
 * skipping j == tidx[i].
 * ------------------------------------------------------------------------- */
void or_p2p(const or_kernel *kern, int64_t ntp, const int64_t *tidx, const int64_t *roff,
            const int64_t *rbeg, const int64_t *rend, const double *pos, const double *mass,
            double *phi, double *acc) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t t = 0; t < ntp; ++t) {
    const int64_t i = tidx[t];
    double f = 0.0, a[3] = {0.0, 0.0, 0.0};
    for (int64_t e = roff[t]; e < roff[t + 1]; ++e)
      for (int64_t j = rbeg[e]; j < rend[e]; ++j) {
        if (j == i) continue;
        double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
               dz = pos[3 * i + 2] - pos[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz), F = or_force_factor(kern, r);
        f -= mass[j] * or_g(kern, r);
        a[0] -= mass[j] * dx * F; a[1] -= mass[j] * dy * F; a[2] -= mass[j] * dz * F;
      }
    phi[t] = f;
    for (int d = 0; d < 3; ++d) acc[3 * t + d] = a[d];
  }
}

/* All-pairs direct sum for the targets tidx[] against all n particles. */
void or_direct(const or_kernel *kern, int64_t nt, const int64_t *tidx, int64_t n, const double *pos,
               const double *mass, double *phi, double *acc) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t t = 0; t < nt; ++t) {
    const int64_t i = tidx[t];
    double f = 0.0, a[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
             dz = pos[3 * i + 2] - pos[3 * j + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz), F = or_force_factor(kern, r);
      f -= mass[j] * or_g(kern, r);
      a[0] -= mass[j] * dx * F; a[1] -= mass[j] * dy * F; a[2] -= mass[j] * dz * F;
    }
    phi[t] = f;
    for (int d = 0; d < 3; ++d) acc[3 * t + d] = a[d];
  }
}

/* Batched small dense products y_b = T x_b for rows x_b of length m, used by
 * the paper-form child-to-parent and parent-to-child passes. */
void or_apply(int m, int64_t nrow, const double *T, int transpose, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nrow; ++b)
    for (int p = 0; p < m; ++p) {
      double s = 0.0;
      for (int q = 0; q < m; ++q) s += (transpose ? T[q * m + p] : T[p * m + q]) * x[b * m + q];
      y[b * m + p] = s;
    }
}

/* Near field of every particle of each leaf: leaf k holds particles
 * [lbeg[k], lend[k]) and its near zone is the ranges e in roff[k] .. roff[k+1].
 * Writes phi/acc at the particles' (sorted) indices. */
void or_p2p_leaves(const or_kernel *kern, int64_t nleaf, const int64_t *lbeg, const int64_t *lend,
                   const int64_t *roff, const int64_t *rbeg, const int64_t *rend,
                   const double *pos, const double *mass, double *phi, double *acc) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < nleaf; ++k)
    for (int64_t i = lbeg[k]; i < lend[k]; ++i) {
      double f = 0.0, a[3] = {0.0, 0.0, 0.0};
      for (int64_t e = roff[k]; e < roff[k + 1]; ++e)
        for (int64_t j = rbeg[e]; j < rend[e]; ++j) {
          if (j == i) continue;
          double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                 dz = pos[3 * i + 2] - pos[3 * j + 2];
          const double r = sqrt(dx * dx + dy * dy + dz * dz), F = or_force_factor(kern, r);
          f -= mass[j] * or_g(kern, r);
          a[0] -= mass[j] * dx * F; a[1] -= mass[j] * dy * F; a[2] -= mass[j] * dz * F;
        }
      phi[i] += f;
      for (int d = 0; d < 3; ++d) acc[3 * i + d] += a[d];
    }
}
