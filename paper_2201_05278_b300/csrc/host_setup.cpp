// Host FP64 set-up (weights, dt, damping, Kaiser-sinc, Ricker).
#include "host_setup.h"

#include <cmath>

namespace sw {

namespace {
// (M!)^2 / ((M-j)! (M+j)!) = prod_{i=1..j} (M-j+i)/(M+i), formed as a product of
// ratios so no factorial overflows.
double factorial_ratio(int M, int j) {
  double r = 1.0;
  for (int i = 1; i <= j; ++i) r *= double(M - j + i) / double(M + i);
  return r;
}
}  // namespace

// Central weights of radius M (closed form of the standard centred formulas):
//   v_j = 2 (-1)^(j+1) (M!)^2 / (j^2 (M-j)! (M+j)!),  v_0 = -2 sum_j v_j.
void fd_second_weights(int order, double* v) {
  const int M = order / 2;
  double s = 0.0;
  for (int j = 1; j <= M; ++j) {
    double sign = (j % 2 == 1) ? 1.0 : -1.0;
    v[j] = 2.0 * sign * factorial_ratio(M, j) / double(j * j);
    s += v[j];
  }
  v[0] = -2.0 * s;
}

//   w_j = 2 (-1)^(j+1) (M!)^2 / (j (M-j)! (M+j)!), for the 1/(2h) prefactor.
void fd_first_weights(int order, double* w) {
  const int M = order / 2;
  w[0] = 0.0;
  for (int j = 1; j <= M; ++j) {
    double sign = (j % 2 == 1) ? 1.0 : -1.0;
    w[j] = 2.0 * sign * factorial_ratio(M, j) / double(j);
  }
}

double stencil_abs_sum(int order) {
  double v[kMaxRadius + 1];
  fd_second_weights(order, v);
  double a = std::fabs(v[0]);
  for (int j = 1; j <= order / 2; ++j) a += 2.0 * std::fabs(v[j]);
  return a;
}

double critical_dt(int ndim, int order, const double* h, double c_max) {
  const double A = stencil_abs_sum(order);
  double s = 0.0;
  for (int i = 0; i < ndim; ++i) s += A / (h[i] * h[i]);
  return 2.0 / (c_max * std::sqrt(s));
}

void damping_coefficients(double alpha, int degree, double dt, int64_t d2, double* a, double* e) {
  double d = std::sqrt(double(d2));
  double dp = 1.0;
  for (int i = 0; i < degree; ++i) dp *= d;
  *e = (d2 == 0) ? 0.0 : alpha * dp * dt;
  *a = 1.0 / (1.0 + *e);
}

double bessel_i0(double x) {
  // I0(x) = sum_k ((x/2)^k / k!)^2; terms are positive, stop at relative 1e-17.
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}

// Kaiser parameter b for half-width r.  The paper gives b = 6.31 for r = 4;
// the rest of this table is a parameter choice for the other radii.
double kaiser_b(int r) {
  static const double table[kMaxRadius + 1] = {0.0,  1.24, 2.94,  4.53,  6.31, 7.91,
                                               9.42, 10.95, 12.53, 14.09, 14.18};
  return (r >= 1 && r <= kMaxRadius) ? table[r] : 0.0;
}

void kaiser_sinc_weights(double s, int r, int64_t* first, double* w) {
  const double b = kaiser_b(r);
  const double i0b = bessel_i0(b);
  const double base = std::floor(s);
  *first = int64_t(base) - r + 1;
  for (int j = 0; j < 2 * r; ++j) {
    const double x = double(*first + j) - s;  // node minus point
    double win = 0.0;
    if (std::fabs(x) <= double(r)) {
      const double q = x / double(r);
      win = bessel_i0(b * std::sqrt(std::fmax(0.0, 1.0 - q * q))) / i0b;
    }
    double sn;
    if (x == 0.0)
      sn = 1.0;
    else if (x == std::floor(x))
      sn = 0.0;  // sinc vanishes at nonzero integers
    else
      sn = std::sin(M_PI * x) / (M_PI * x);
    w[j] = win * sn;
  }
}

void ricker(double f_peak, double t0, double dt, int nt, float* out) {
  for (int n = 0; n < nt; ++n) {
    const double tau = double(n) * dt - t0;
    const double a = (M_PI * f_peak * tau) * (M_PI * f_peak * tau);
    out[n] = float((1.0 - 2.0 * a) * std::exp(-a));
  }
}

}  // namespace sw
