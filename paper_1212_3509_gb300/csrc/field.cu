// Stray field from analytic derivative factors: h_d = -grad phi at the
// collocation points without finite differences.
//
// In the Kronecker form of phi (Cor. 3, Eq. kron_operator) the collocation
// point enters each 1D factor only through the limits of its cell integral,
// T[d] = int_{a_d}^{b_d} f(x) dx with a_d, b_d = (d -+ 1/2) hh, so d/dxi_p acts
// on the axis-p factor alone and replaces it by f(b_d) - f(a_d):
//   E (f = exp(-tau^2 x^2))    ->  dE[d] = -2 tau^2 F[d]            (odd in d)
//   F (f = x exp(-tau^2 x^2))  ->  dF[d] = b e^{-tau^2 b^2} - a e^{-tau^2 a^2}   (even)
// With the domain scaled by s (Sec. 3.4) the derivative with respect to the
// physical coordinate carries 1/s, folded into the generators here, so the
// chains that apply phi (c s omega_k on the third axis) give the field.
#include <cmath>

#include "internal.h"

namespace demag {

// gend[k][type][p][e], type 0 = dE / s, type 1 = dF / s, from the nodes and
// the F generators already in gen64.  dF for |d| >= 1 is written
// exp(-tau^2 a^2) (hh + b expm1(-2 |d| tau^2 hh^2)), free of the cancellation
// of the two exponentials.
__global__ void deriv_generators_kernel(int M, int glen, GridInfo g, double inv_s, const double* nodes,
                                        const double* gen64, double* gend) {
  const long total = (long)M * 2 * 3 * glen;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const int e = (int)(idx % glen);
    long rest = idx / glen;
    const int p = (int)(rest % 3);
    rest /= 3;
    const int type = (int)(rest % 2);
    const int k = (int)(rest / 2);
    const int n = g.n[p];
    double val = 0.0;
    if (e < 2 * n - 1) {
      const double tau = nodes[M + k];
      const double t2 = tau * tau;
      if (type == 0) {
        // F of the same (k, axis, d): type 1 in gen64
        val = -2.0 * t2 * gen64[(((long)k * 2 + 1) * 3 + p) * glen + e];
      } else {
        const int d = e - (n - 1);
        const int ad = d < 0 ? -d : d;
        const double hh = g.hh[p];
        if (ad == 0) {
          val = hh * exp(-0.25 * t2 * hh * hh);
        } else {
          const double a = ((double)ad - 0.5) * hh, b = a + hh;
          val = exp(-t2 * a * a) * (hh + b * expm1(-2.0 * ad * t2 * hh * hh));
        }
      }
      val *= inv_s;
    }
    gend[idx] = val;
  }
}

demag_status ensure_field_generators(demag_plan* P, cudaStream_t st) {
  if (P->gend) return DEMAG_OK;
  const long total = (long)P->M * 6 * P->glen;
  DEMAG_CUDA(P, cudaMalloc(&P->gend, sizeof(double) * total));
  GridInfo g;
  for (int p = 0; p < 3; ++p) {
    g.n[p] = P->n[p];
    g.hh[p] = P->hh[p];
  }
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  DEMAG_LAUNCH(P, kFamSetup, st,
               deriv_generators_kernel<<<blocks, 256, 0, st>>>(P->M, P->glen, g, 1.0 / P->s, P->nodes, P->gen64,
                                                               P->gend));
  DEMAG_LAUNCHED(P, "deriv_generators_kernel");
  return DEMAG_OK;
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_stray_field_exact(demag_plan* P, const float* m, float* hd, demag_precision prec,
                                                void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_stray_field_exact: plan is NULL");
  if (!m || !hd) return set_error(P, DEMAG_EINVAL, "demag_stray_field_exact: NULL pointer");
  demag_status u = require_uniform(P, "demag_stray_field_exact");  // derivative generators are Toeplitz
  if (u != DEMAG_OK) return u;
  if ((int)prec < 0 || (int)prec > (int)DEMAG_BF16X3)
    return set_error(P, DEMAG_EINVAL, "demag_stray_field_exact: unknown precision %d", (int)prec);
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) return tc_field(P, m, hd, prec, st);
  return simt_field(P, m, hd, prec, st);
}
