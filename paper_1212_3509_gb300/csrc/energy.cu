// Stray field, demag energy and its gradient.
//
// h_d = -grad phi (Sec. 1, the definition before Eq. poisson).  The energy
// study after Alg. 2 discretises the stray field and the energy "second
// order" (footnote there) without naming the stencil; this file uses central
// differences inside, 3-point one-sided differences at the first and last
// cell of each axis (two-point when n_p = 2, zero when n_p = 1), and the
// midpoint rule E = -1/2 h1 h2 h3 sum_i m_i . h_d,i.  With phi = P m,
// dE/dm = 1/2 h1 h2 h3 (D P m + P^T D^T m).
#include "internal.h"

namespace demag {

struct FDGrid {
  int n[3];
  float inv2h[3];  // 1 / (2 h_p)
};

// Coefficient D_p[i][j] of the 1D derivative matrix (row i = output cell).
__device__ __forceinline__ float fd_coef(int i, int j, int n, float inv2h) {
  if (n == 1) return 0.f;
  if (n == 2) return (j == 1 ? 2.f : -2.f) * inv2h;  // (phi1 - phi0) / h
  if (i == 0) return j == 0 ? -3.f * inv2h : j == 1 ? 4.f * inv2h : j == 2 ? -inv2h : 0.f;
  if (i == n - 1) return j == n - 1 ? 3.f * inv2h : j == n - 2 ? -4.f * inv2h : j == n - 3 ? inv2h : 0.f;
  return j == i + 1 ? inv2h : j == i - 1 ? -inv2h : 0.f;
}

// transpose: sum_i D[i][c] g[i]
__device__ __forceinline__ float fdT_apply(const float* g, long idx, int c, int n, long st, float inv2h) {
  float acc = 0.f;
  int lo = c - 2 < 0 ? 0 : c - 2, hi = c + 2 > n - 1 ? n - 1 : c + 2;
  for (int i = lo; i <= hi; ++i) acc += fd_coef(i, c, n, inv2h) * g[idx + (long)(i - c) * st];
  return acc;
}

// The same stencils written out: central inside, one-sided at the two end cells
__device__ __forceinline__ float fd_fast(const float* f, long idx, int c, int n, long st, float inv2h) {
  if (c > 0 && c < n - 1) return inv2h * (f[idx + st] - f[idx - st]);
  if (n == 1) return 0.f;
  if (n == 2) return 2.f * inv2h * (c == 0 ? f[idx + st] - f[idx] : f[idx] - f[idx - st]);
  if (c == 0) return inv2h * (-3.f * f[idx] + 4.f * f[idx + st] - f[idx + 2 * st]);
  return inv2h * (3.f * f[idx] - 4.f * f[idx - st] + f[idx - 2 * st]);
}

// transpose: away from the ends (3 <= c <= n - 4) only the central rows c - 1 and c + 1 reach
// column c; near the ends the one-sided rows contribute too (general loop)
__device__ __forceinline__ float fdT_fast(const float* g, long idx, int c, int n, long st, float inv2h) {
  if (c >= 3 && c <= n - 4) return inv2h * (g[idx - st] - g[idx + st]);
  return fdT_apply(g, idx, c, n, st, inv2h);
}

// out[p][cell] = scale * (D_p phi)[cell]
__global__ void fd_gradient_kernel(FDGrid g, const float* phi, float* out, float scale) {
  const long N = (long)g.n[0] * g.n[1] * g.n[2];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
    int i1 = (int)(idx % g.n[0]);
    int i2 = (int)((idx / g.n[0]) % g.n[1]);
    int i3 = (int)(idx / ((long)g.n[0] * g.n[1]));
    out[idx] = scale * fd_fast(phi, idx, i1, g.n[0], 1, g.inv2h[0]);
    out[N + idx] = scale * fd_fast(phi, idx, i2, g.n[1], g.n[0], g.inv2h[1]);
    out[2 * N + idx] = scale * fd_fast(phi, idx, i3, g.n[2], (long)g.n[0] * g.n[1], g.inv2h[2]);
  }
}

// out[cell] = sum_p (D_p^T v_p)[cell]
__global__ void fd_adjoint_kernel(FDGrid g, const float* v, float* out) {
  const long N = (long)g.n[0] * g.n[1] * g.n[2];
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
    int i1 = (int)(idx % g.n[0]);
    int i2 = (int)((idx / g.n[0]) % g.n[1]);
    int i3 = (int)(idx / ((long)g.n[0] * g.n[1]));
    out[idx] = fdT_fast(v, idx, i1, g.n[0], 1, g.inv2h[0]) +
               fdT_fast(v + N, idx, i2, g.n[1], g.n[0], g.inv2h[1]) +
               fdT_fast(v + 2 * N, idx, i3, g.n[2], (long)g.n[0] * g.n[1], g.inv2h[2]);
  }
}

// energy += half_vol * sum_cells m . (D phi) (each cell's three products in FP32, cells summed in
// FP64) and, with grad, grad[p][cell] = gscale ((D_p phi)[cell] + ptdtm[p][cell]): the energy and
// its gradient 1/2 h1 h2 h3 (D P m + P^T D^T m) in one pass over phi, m and P^T D^T m
__global__ void energy_grad_kernel(FDGrid g, const float* m, const float* phi, const float* ptdtm, double half_vol,
                                   float gscale, double* energy, float* grad) {
  const long N = (long)g.n[0] * g.n[1] * g.n[2];
  double acc = 0.0;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < N; idx += (long)gridDim.x * blockDim.x) {
    int i1 = (int)(idx % g.n[0]);
    int i2 = (int)((idx / g.n[0]) % g.n[1]);
    int i3 = (int)(idx / ((long)g.n[0] * g.n[1]));
    const float d1 = fd_fast(phi, idx, i1, g.n[0], 1, g.inv2h[0]);
    const float d2 = fd_fast(phi, idx, i2, g.n[1], g.n[0], g.inv2h[1]);
    const float d3 = fd_fast(phi, idx, i3, g.n[2], (long)g.n[0] * g.n[1], g.inv2h[2]);
    acc += (double)fmaf(m[idx], d1, fmaf(m[N + idx], d2, m[2 * N + idx] * d3));
    if (grad) {
      grad[idx] = gscale * (d1 + ptdtm[idx]);
      grad[N + idx] = gscale * (d2 + ptdtm[N + idx]);
      grad[2 * N + idx] = gscale * (d3 + ptdtm[2 * N + idx]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(energy, half_vol * v);
  }
}

static FDGrid fd_grid(const demag_plan* P) {
  FDGrid g;
  for (int p = 0; p < 3; ++p) {
    g.n[p] = P->n[p];
    g.inv2h[p] = (float)(0.5 / P->h[p]);
  }
  return g;
}

static int blocks_for(long count) {
  long b = (count + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

demag_status fd_gradient(demag_plan* P, const float* phi, float* out, float scale, cudaStream_t st) {
  const long N = (long)field_size(P);
  DEMAG_LAUNCH(P, kFamEnergy, st, fd_gradient_kernel<<<blocks_for(N), 256, 0, st>>>(fd_grid(P), phi, out, scale));
  DEMAG_LAUNCHED(P, "fd_gradient_kernel");
  return DEMAG_OK;
}

void energy_destroy(demag_plan* P) {
  cudaFree(P->ews);
  P->ews = nullptr;
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_stray_field(demag_plan* P, const float* phi, float* hd, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_stray_field: plan is NULL");
  if (!phi || !hd) return set_error(P, DEMAG_EINVAL, "demag_stray_field: NULL pointer");
  demag_status u = require_uniform(P, "demag_stray_field");  // uniform difference stencils
  if (u != DEMAG_OK) return u;
  return fd_gradient(P, phi, hd, -1.f, (cudaStream_t)stream);
}

extern "C" demag_status demag_energy(demag_plan* P, const float* m, double* energy, float* grad,
                                     demag_precision prec, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy: plan is NULL");
  if (!m || !energy) return set_error(P, DEMAG_EINVAL, "demag_energy: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy");  // uniform difference stencils and cell volume
  if (u != DEMAG_OK) return u;
  cudaStream_t st = (cudaStream_t)stream;
  const long N = (long)field_size(P);
  if (!P->ews) DEMAG_CUDA(P, cudaMalloc(&P->ews, sizeof(float) * 5 * N));
  float* phi = P->ews;
  float* dtm = phi + N;
  float* ptdtm = dtm + N;
  demag_status s = full_forward(P, m, phi, prec, st);
  if (s != DEMAG_OK) return s;
  const double vol = P->h[0] * P->h[1] * P->h[2];
  if (grad) {
    // P^T (D^T m) first, then one pass for the energy and grad = 1/2 V (D P m + P^T D^T m)
    DEMAG_LAUNCH(P, kFamEnergy, st, fd_adjoint_kernel<<<blocks_for(N), 256, 0, st>>>(fd_grid(P), m, dtm));
    DEMAG_LAUNCHED(P, "fd_adjoint_kernel");
    s = full_adjoint(P, dtm, ptdtm, prec, st);
    if (s != DEMAG_OK) return s;
  }
  DEMAG_CUDA(P, cudaMemsetAsync(energy, 0, sizeof(double), st));
  DEMAG_LAUNCH(P, kFamEnergy, st,
               energy_grad_kernel<<<blocks_for(N), 256, 0, st>>>(fd_grid(P), m, phi, grad ? ptdtm : nullptr,
                                                                 0.5 * vol, (float)(0.5 * vol), energy, grad));
  DEMAG_LAUNCHED(P, "energy_grad_kernel");
  return DEMAG_OK;
}
