// Factor matrices of the Kronecker operator on a non-uniform tensor grid.
//
// Sec. 3.1 partitions each axis into arbitrary sub-intervals I_j = [y_j, y_{j+1}]
// with collocation at their midpoints xi_i; Eq. sep_integrands and Cor. 3
// (Eq. kron_operator) then give per node tau_k the dense factors
//   E[i][j] = int_{I_j} exp(-tau^2 (xi_i - y)^2) dy = int_a^b exp(-tau^2 x^2) dx,
//   F[i][j] = int_{I_j} (xi_i - y) exp(-tau^2 (xi_i - y)^2) dy = int_a^b x exp(-tau^2 x^2) dx,
// a = xi_i - y_{j+1} < b = xi_i - y_j, in coordinates scaled by the longest
// domain edge s.  They are no longer Toeplitz (the cell widths differ), so the
// plan keeps them as full matrices in the layout of the dense factor tables;
// the full-format chains then run unchanged.
#include <cmath>

#include "internal.h"

namespace demag {

// int_a^b exp(-tau^2 x^2) dx, a < b.  Mirrored to b > 0; when both limits are
// in the tail (tau a >= 1/2) the erf difference is taken as
// exp(-tau^2 a^2) (erfcx(tau a) - exp(-tau^2 (b - a)(b + a)) erfcx(tau b)),
// the same number without cancellation.
__device__ double cell_integral_E(double tau, double a, double b) {
  if (b <= 0.0) {
    const double t = a;
    a = -b;
    b = -t;
  }
  const double ta = tau * a, tb = tau * b;
  double diff;
  if (ta < 0.5)
    diff = erf(tb) - erf(ta);
  else
    diff = exp(-ta * ta) * (erfcx(ta) - exp(-(tb - ta) * (tb + ta)) * erfcx(tb));
  return 0.5 * 1.7724538509055160273 / tau * diff;
}

// int_a^b x exp(-tau^2 x^2) dx, a < b: odd under (a, b) -> (-b, -a); for
// 0 <= a written exp(-tau^2 a^2) (-expm1(-tau^2 (b - a)(b + a))) / (2 tau^2).
__device__ double cell_integral_F(double tau, double a, double b) {
  double sgn = 1.0;
  if (b <= 0.0) {
    const double t = a;
    a = -b;
    b = -t;
    sgn = -1.0;
  }
  const double t2 = tau * tau;
  double v;
  if (a >= 0.0)
    v = exp(-t2 * a * a) * (-expm1(-t2 * (b - a) * (b + a))) / (2.0 * t2);
  else
    v = (exp(-t2 * a * a) - exp(-t2 * b * b)) / (2.0 * t2);
  return sgn * v;
}

// fac[k][type][block of axis p][i][j] (blocks at 0, off1, off2 of a group of
// tgroup entries); y holds the scaled edges of the three axes at 0, yoff1,
// yoff2.  The diagonal (the collocation point's own cell, symmetric about it)
// is E = sqrt(pi)/tau erf(tau w/2), F = 0 exactly.
__global__ void nonuniform_factor_kernel(int M, int n0, int n1, int n2, size_t tgroup, size_t off1, size_t off2,
                                         int yoff1, int yoff2, const double* nodes, const double* y, double* fac) {
  const size_t total = (size_t)M * 2 * tgroup;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t e = idx % tgroup;
    const size_t kt = idx / tgroup;  // k * 2 + type
    const int type = (int)(kt & 1), k = (int)(kt >> 1);
    int n;
    size_t local;
    const double* yp;
    if (e < off1) { n = n0; local = e; yp = y; }
    else if (e < off2) { n = n1; local = e - off1; yp = y + yoff1; }
    else { n = n2; local = e - off2; yp = y + yoff2; }
    const int i = (int)(local / n), j = (int)(local % n);
    const double tau = nodes[M + k];
    double v;
    if (i == j) {
      v = type ? 0.0 : 1.7724538509055160273 / tau * erf(0.5 * tau * (yp[i + 1] - yp[i]));
    } else {
      const double xi = 0.5 * (yp[i] + yp[i + 1]);
      const double a = xi - yp[j + 1], b = xi - yp[j];
      v = type ? cell_integral_F(tau, a, b) : cell_integral_E(tau, a, b);
    }
    fac[idx] = v;
  }
}

demag_status require_uniform(demag_plan* P, const char* what) {
  if (P && P->nonuniform)
    return set_error(P, DEMAG_EUNSUPPORTED, "%s: needs a uniform grid (this plan has non-uniform cells)", what);
  return DEMAG_OK;
}

}  // namespace demag
