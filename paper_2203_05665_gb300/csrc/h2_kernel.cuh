// The kernel functions g(x, y) of Section 1 evaluated by the set-up kernels:
// the Laplace kernel 1 / (4 pi r) and the real and imaginary parts of the
// Helmholtz kernel e^{i kappa r} / (4 pi r), r = |x - y|: cos(kappa r) /
// (4 pi r) and sin(kappa r) / (4 pi r) (smooth, kappa / (4 pi) at r = 0).
// The Helmholtz matrix is assembled as two real H^2 matrices with these
// kernels (same trees, bases and quadrature).
#pragma once

#include "h2_internal.hpp"

namespace h2 {

constexpr double kInv4PiK = 0.079577471545947667884441881686257181;

// r and 1 / (4 pi r) are formed once, the same way for every kind, and
// kappa = 0 takes the limits e^{i 0 r} = 1 exactly (the real part is the
// Laplace kernel, the imaginary part vanishes) without calling cos or sin
__device__ __forceinline__ double kernel_value(KernelFn kf, const double *x, const double *y) {
  const double d0 = x[0] - y[0], d1 = x[1] - y[1], d2 = x[2] - y[2];
  const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  const double g = kInv4PiK / r;
  if (kf.kind == kKernelLaplace) return g;
  if (kf.kind == kKernelHelmholtzRe) return kf.kappa == 0.0 ? g : cos(kf.kappa * r) * g;
  if (kf.kappa == 0.0) return 0.0;
  return r > 0.0 ? sin(kf.kappa * r) * g : kf.kappa * kInv4PiK;
}

}  // namespace h2
