/*
 * Radial Green functions handed to the solver and to the FP64 oracle through
 * their user-kernel interfaces (double g(double r, void *ctx)). Test input,
 * like the particle sets: both sides call the same functions, neither shares
 * any other code. Each comes with its exact derivative for the oracle.
 */
#include <math.h>

/* erf(r / a) / r: the potential of a unit Gaussian charge of width a
 * (density exp(-r^2/a^2) / (pi^{3/2} a^3)); ctx points to a. Near r = 0 the
 * Taylor series of erf(x)/x keeps full precision. */
double hpm_test_erf_g(double r, void *ctx) {
  const double a = *(const double *)ctx, x = r / a, c = 2.0 / (a * sqrt(M_PI));
  if (x < 1e-4) return c * (1.0 - x * x / 3.0 + x * x * x * x / 10.0);
  return erf(x) / r;
}

double hpm_test_erf_dg(double r, void *ctx) {
  const double a = *(const double *)ctx, x = r / a, c = 2.0 / (a * sqrt(M_PI));
  if (x < 1e-4) return c * (-2.0 * x / 3.0 + 4.0 * x * x * x / 10.0) / a;
  return (c * exp(-x * x) - erf(x) / r) / r;
}

/* Plummer 1 / sqrt(r^2 + eps^2) through the same interface; ctx points to eps. */
double hpm_test_plummer_g(double r, void *ctx) {
  const double e = *(const double *)ctx;
  return 1.0 / sqrt(r * r + e * e);
}

double hpm_test_plummer_dg(double r, void *ctx) {
  const double e = *(const double *)ctx, s2 = r * r + e * e;
  return -r / (s2 * sqrt(s2));
}
