// Host FP64 set-up of the solver: FD weights, stable time step, damping
// coefficients, Kaiser-windowed sinc weights, Ricker samples.
#pragma once

#include <cstdint>
#include <vector>

namespace sw {

constexpr int kMaxRadius = 10;  // space order 20

// Eq. 9: v[0..r] with h^2 f'' ~ v0 f0 + sum_j v_j (f_j + f_-j), r = order/2.
void fd_second_weights(int order, double* v);
// Eq. 10: w[1..r] with f' ~ (1/2h) sum_j w_j (f_j - f_-j); w[0] set to 0.
void fd_first_weights(int order, double* w);
// |v0| + 2 sum |v_j|: one axis' share of the coefficient sum of Eq. 8.
double stencil_abs_sum(int order);
// Eq. 8: dt <= 2 / (c_max sqrt(sum_axes A / h^2)).
double critical_dt(int ndim, int order, const double* h, double c_max);

// Damping coefficients for a squared distance d2 (cells^2) to the physical
// domain: e = eta dt = alpha d^p dt and a = 1/(1+e) (Eq. 4, 7).
void damping_coefficients(double alpha, int degree, double dt, int64_t d2, double* a, double* e);

// Sec. 2.4: modified Bessel I0 (power series), Kaiser parameter b(r), and the
// 2r separable weights of a point at cell coordinate s.
double bessel_i0(double x);
double kaiser_b(int r);
void kaiser_sinc_weights(double s, int r, int64_t* first, double* w);

void ricker(double f_peak, double t0, double dt, int nt, float* out);

}  // namespace sw
