// Tensor-train arithmetic of App. C: conversions of CP and Tucker tensors to
// 3D tensor trains and the Hadamard (element-wise) product of two trains.
//
// A 3D train is a[i1,i2,i3] = sum_{a1,a2} G1(i1,a1) G2(a1,i2,a2) G3(a2,i3)
// (Eq. tt_3d_1).  Layouts as the TT application: G1 [r1][n1], G2 [r1 r2][n2]
// with row a1 r2 + a2, G3 [r2][n3], three components one after another.
//
// * Tucker [[C; V1, V2, V3]] -> TT by multiplying the second factor into the
//   core (the remark after Eq. tt_3d_2): ranks (r1, r3), G1 = V1, G3 = V3,
//   G2(a1, i2, a3) = sum_a2 C[a3][a2][a1] V2[a2][i2].
// * CP sum_l lambda_l u1_l o u2_l o u3_l -> TT with ranks (r, r): G1 = U1,
//   G3 = U3, G2(a1, i2, a2) = delta_{a1 a2} lambda_a1 U2[a1][i2].
// * Hadamard product: the cores multiply slice by slice as Kronecker
//   products, so the ranks multiply: C1 row a rb1 + b = A1[a] B1[b] (per i1),
//   C2 row (a1 rb1 + b1) (ra2 rb2) + (a2 rb2 + b2) = A2[a1 ra2 + a2] B2[b1 rb2 + b2],
//   C3 row a2 rb2 + b2 = A3[a2] B3[b2].
// Every output element is independent: grid-stride element kernels, FP32
// (the Tucker core product accumulates r2 terms in FP32).
#include "internal.h"

namespace demag {

static int arith_blocks(long total) {
  long b = (total + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152L * 32 ? 152L * 32 : b));
}

// G2[q][(a1 r3 + a3)][i2] = sum_a2 C[q][a3][a2][a1] V2[q][a2][i2]
__global__ void tucker_tt_core_kernel(int r1, int r2, int r3, int n2, long vq_stride, const float* C, const float* V2,
                                      float* G2) {
  const long per = (long)r1 * r3 * n2, total = 3 * per;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / per);
    const long e = idx - q * per;
    const int i2 = (int)(e % n2);
    const int row = (int)(e / n2);
    const int a1 = row / r3, a3 = row % r3;
    const float* c = C + (long)q * r1 * r2 * r3 + (long)a3 * r2 * r1 + a1;
    const float* v = V2 + q * vq_stride + i2;
    float acc = 0.f;
    for (int a2 = 0; a2 < r2; ++a2) acc = fmaf(c[(long)a2 * r1], v[(long)a2 * n2], acc);
    G2[idx] = acc;
  }
}

// out[q][row][i] = in[q][row][i] for the rows of one factor block (strided input blocks)
__global__ void copy_rows_kernel(long per, long in_qstride, const float* in, float* out) {
  const long total = 3 * per;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / per);
    out[idx] = in[q * in_qstride + (idx - q * per)];
  }
}

// G2[q][(a1 r + a2)][i2] = (a1 == a2) lambda[q][a1] U2[q][a1][i2]
__global__ void cp_tt_core_kernel(int r, int n2, long uq_stride, const float* lambda, const float* U2, float* G2) {
  const long per = (long)r * r * n2, total = 3 * per;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / per);
    const long e = idx - q * per;
    const int i2 = (int)(e % n2);
    const int row = (int)(e / n2);
    const int a1 = row / r, a2 = row % r;
    G2[idx] = a1 == a2 ? lambda[q * r + a1] * U2[q * uq_stride + (long)a1 * n2 + i2] : 0.f;
  }
}

// C[q][(a ra_in + ...)]: the Kronecker product of the rank indices of one core pair.
// Core k of a train has rows (x, y) with x < px, y < py (px = 1 for G1, py = 1 for G3);
// the product core has rows ((xa xb), (ya yb)) = ((xa pxb + xb) (pya pyb) + (ya pyb + yb)).
__global__ void tt_hadamard_kernel(int n, int pxa, int pya, int pxb, int pyb, const float* A, const float* B,
                                   float* C) {
  const long rows = (long)pxa * pxb * pya * pyb, per = rows * n, total = 3 * per;
  const long ra = (long)pxa * pya * n, rb = (long)pxb * pyb * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int q = (int)(idx / per);
    const long e = idx - q * per;
    const int i = (int)(e % n);
    const long row = e / n;
    const int ycol = (int)(row % ((long)pya * pyb)), xrow = (int)(row / ((long)pya * pyb));
    const int xa = xrow / pxb, xb = xrow % pxb, ya = ycol / pyb, yb = ycol % pyb;
    C[idx] = A[q * ra + ((long)xa * pya + ya) * n + i] * B[q * rb + ((long)xb * pyb + yb) * n + i];
  }
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_tucker_to_tt(demag_plan* P, const int r[3], const float* core, const float* V,
                                           float* G1, float* G2, float* G3, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_tucker_to_tt: plan is NULL");
  if (!r || !core || !V || !G1 || !G2 || !G3) return set_error(P, DEMAG_EINVAL, "demag_tucker_to_tt: NULL pointer");
  for (int p = 0; p < 3; ++p)
    if (r[p] < 1) return set_error(P, DEMAG_EINVAL, "demag_tucker_to_tt: ranks must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const long qstride = (long)r[0] * n1 + (long)r[1] * n2 + (long)r[2] * n3;  // V blocks (q, p)
  const long p1 = (long)r[0] * n1, p3 = (long)r[2] * n3;
  DEMAG_LAUNCH(P, kFamMisc, st, copy_rows_kernel<<<arith_blocks(3 * p1), 256, 0, st>>>(p1, qstride, V, G1));
  DEMAG_LAUNCHED(P, "copy_rows_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               copy_rows_kernel<<<arith_blocks(3 * p3), 256, 0, st>>>(p3, qstride, V + p1 + (long)r[1] * n2, G3));
  DEMAG_LAUNCHED(P, "copy_rows_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               tucker_tt_core_kernel<<<arith_blocks(3L * r[0] * r[2] * n2), 256, 0, st>>>(r[0], r[1], r[2], n2, qstride,
                                                                                          core, V + p1, G2));
  DEMAG_LAUNCHED(P, "tucker_tt_core_kernel");
  return DEMAG_OK;
}

extern "C" demag_status demag_cp_to_tt(demag_plan* P, int r, const float* lambda, const float* U, float* G1,
                                       float* G2, float* G3, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_cp_to_tt: plan is NULL");
  if (!lambda || !U || !G1 || !G2 || !G3) return set_error(P, DEMAG_EINVAL, "demag_cp_to_tt: NULL pointer");
  if (r < 1) return set_error(P, DEMAG_EINVAL, "demag_cp_to_tt: r must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const long qstride = (long)r * (n1 + n2 + n3);  // U blocks (q, p), each [r][n_p]
  const long p1 = (long)r * n1, p3 = (long)r * n3;
  DEMAG_LAUNCH(P, kFamMisc, st, copy_rows_kernel<<<arith_blocks(3 * p1), 256, 0, st>>>(p1, qstride, U, G1));
  DEMAG_LAUNCHED(P, "copy_rows_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               copy_rows_kernel<<<arith_blocks(3 * p3), 256, 0, st>>>(p3, qstride, U + p1 + (long)r * n2, G3));
  DEMAG_LAUNCHED(P, "copy_rows_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               cp_tt_core_kernel<<<arith_blocks(3L * r * r * n2), 256, 0, st>>>(r, n2, qstride, lambda, U + p1, G2));
  DEMAG_LAUNCHED(P, "cp_tt_core_kernel");
  return DEMAG_OK;
}

extern "C" demag_status demag_tt_hadamard(demag_plan* P, const int ra[2], const float* A1, const float* A2,
                                          const float* A3, const int rb[2], const float* B1, const float* B2,
                                          const float* B3, float* C1, float* C2, float* C3, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_tt_hadamard: plan is NULL");
  if (!ra || !rb || !A1 || !A2 || !A3 || !B1 || !B2 || !B3 || !C1 || !C2 || !C3)
    return set_error(P, DEMAG_EINVAL, "demag_tt_hadamard: NULL pointer");
  if (ra[0] < 1 || ra[1] < 1 || rb[0] < 1 || rb[1] < 1)
    return set_error(P, DEMAG_EINVAL, "demag_tt_hadamard: ranks must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const long t1 = 3L * ra[0] * rb[0] * n1, t2 = 3L * ra[0] * rb[0] * ra[1] * rb[1] * n2, t3 = 3L * ra[1] * rb[1] * n3;
  DEMAG_LAUNCH(P, kFamMisc, st,
               tt_hadamard_kernel<<<arith_blocks(t1), 256, 0, st>>>(n1, ra[0], 1, rb[0], 1, A1, B1, C1));
  DEMAG_LAUNCHED(P, "tt_hadamard_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               tt_hadamard_kernel<<<arith_blocks(t2), 256, 0, st>>>(n2, ra[0], ra[1], rb[0], rb[1], A2, B2, C2));
  DEMAG_LAUNCHED(P, "tt_hadamard_kernel");
  DEMAG_LAUNCH(P, kFamMisc, st,
               tt_hadamard_kernel<<<arith_blocks(t3), 256, 0, st>>>(n3, ra[1], 1, rb[1], 1, A3, B3, C3));
  DEMAG_LAUNCHED(P, "tt_hadamard_kernel");
  return DEMAG_OK;
}
