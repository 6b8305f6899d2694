// Demag energy of a Tucker magnetization from its potential in Tucker form,
// without forming a full tensor (Alg. 2 and the energy study after it).
//
// m^(q) = [[G^(q); V^(q,1), V^(q,2), V^(q,3)]] (Eq. tucker_rep) and
// phi = sum_t w_t [[C_t; W_t1, W_t2, W_t3]]: either the terms (k, q') of the
// Tucker application (core G^(q'), factors T_{k,q',p} V^(q',p), weight
// c s omega_k; Eq. kron_eval_tuck) or one Tucker tensor (the approximate sum
// of Alg. 2).  The stray field is -D phi with the second-order stencils of
// energy.cu; along axis q the difference acts on the factors of that axis
// only, so with W'_tp = D_q W_tp (p = q) or W_tp (p != q)
//   E = 1/2 h1 h2 h3 sum_q sum_t w_t < m^(q), [[C_t; W'_t1, W'_t2, W'_t3]] >.
// The inner product of two Tucker tensors contracts the cores through the
// factor Grams M_p = V^(q,p)^T W'_tp:
//   <[[G; V]], [[C; W']]> = sum_{a,b} G[a] C[b] prod_p M_p[a_p][b_p].
// One block per (term, component): the Grams in shared memory, the core
// contraction mode by mode through a global workspace, FP64 throughout from
// the FP32 factors; the per-block values are summed in a fixed order.
#include "internal.h"

namespace demag {

constexpr int kEnMaxRank = 64;
// static shared memory of the energy kernels: the two [64][33] tiles of block_gram (float, or
// double for the FP64 Tucker energy) and a 32-double reduction buffer
template <typename T>
constexpr size_t en_static_smem() { return 2 * 64 * 33 * sizeof(T) + 32 * sizeof(double); }
constexpr size_t kEnStaticSmem = en_static_smem<float>();

__device__ __forceinline__ double en_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename F>
struct EnTuckerT {
  int n[3];
  double inv2h[3];   // 1 / (2 h_p)
  int r[3];          // multilinear ranks of m
  const F* G;        // [3][r3][r2][r1]
  const F* V;        // blocks (q, p), each [r_p][n_p]
  int s[3];          // ranks of every phi term
  const F* C;        // term cores [s3][s2][s1]: C + (core_by_q ? t % 3 : 0) * s1 s2 s3
  int core_by_q;
  const F* W[3];     // term t, mode p: rows W[p] + t * s_p * n_p
  const F* w;        // term weights (NULL: 1)
  int T;             // number of terms
  double* ws;        // per block r1 s3 (s2 + r2) doubles
  double* part;      // [T][3]
};
using EnTucker = EnTuckerT<float>;

// (D w)[i] of one factor row with the second-order stencils (central inside,
// 3-point one-sided at the ends, two-point for n = 2, zero for n = 1)
template <typename F>
__device__ __forceinline__ double fd_row(const F* w, int i, int n, double inv2h) {
  if (n == 1) return 0.0;
  if (n == 2) return 2.0 * inv2h * ((double)w[1] - (double)w[0]);
  if (i == 0) return inv2h * (-3.0 * (double)w[0] + 4.0 * (double)w[1] - (double)w[2]);
  if (i == n - 1) return inv2h * (3.0 * (double)w[n - 1] - 4.0 * (double)w[n - 2] + (double)w[n - 3]);
  return inv2h * ((double)w[i + 1] - (double)w[i - 1]);
}

// Mout[a][b] = sum_i A[a][i] B'[b][i] (B' = D B when deriv) for ra, rb <= 64 rows of length n:
// 32-column tiles of A and B' through shared memory (tA, tB: [64][33]), each of the 256 threads
// a 4 x 4 block of outputs; FP32 factors: FP32 products summed within a tile and FP64 across
// tiles; FP64 factors: FP64 throughout.
template <typename F>
__device__ void block_gram(const F* A, int ra, const F* B, int rb, int n, bool deriv, double inv2h,
                           F* tA, F* tB, double* Mout) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int i0 = 0; i0 < n; i0 += 32) {
    for (int e = threadIdx.x; e < 64 * 32; e += blockDim.x) {
      const int r = e >> 5, c = e & 31, i = i0 + c;
      tA[r * 33 + c] = (r < ra && i < n) ? A[(long)r * n + i] : F(0);
      F bv = F(0);
      if (r < rb && i < n) bv = deriv ? (F)fd_row(B + (long)r * n, i, n, inv2h) : B[(long)r * n + i];
      tB[r * 33 + c] = bv;
    }
    __syncthreads();
    F part[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) part[i][j] = F(0);
#pragma unroll 8
    for (int c = 0; c < 32; ++c) {
      F av[4], bw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = tA[(ty + 16 * i) * 33 + c];
        bw[i] = tB[(tx + 16 * i) * 33 + c];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) part[i][j] = fma(av[i], bw[j], part[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += (double)part[i][j];
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ia = ty + 16 * i, ib = tx + 16 * j;
      if (ia < ra && ib < rb) Mout[ia * rb + ib] = acc[i][j];
    }
}

template <typename F>
__global__ void __launch_bounds__(256) tucker_energy_kernel(const __grid_constant__ EnTuckerT<F> a) {
  extern __shared__ double Mg[];
  __shared__ double red[32];
  __shared__ F tA[64 * 33], tB[64 * 33];
  const int t = blockIdx.x, q = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r1 = a.r[0], r2 = a.r[1], r3 = a.r[2];
  const int s1 = a.s[0], s2 = a.s[1], s3 = a.s[2];
  // 1. Grams M_p [r_p][s_p] at offsets sum_{p' < p} r_p' s_p'
  long voff = (long)q * ((long)r1 * a.n[0] + (long)r2 * a.n[1] + (long)r3 * a.n[2]);
  int moff = 0;
  int mo[3];
  for (int p = 0; p < 3; ++p) {
    const int n = a.n[p], rp = a.r[p], sp = a.s[p];
    mo[p] = moff;
    block_gram(a.V + voff, rp, a.W[p] + (long)t * sp * n, sp, n, p == q, a.inv2h[p], tA, tB, Mg + moff);
    voff += (long)rp * n;
    moff += rp * sp;
  }
  __syncthreads();
  const double *M1 = Mg + mo[0], *M2 = Mg + mo[1], *M3 = Mg + mo[2];
  const F* Ct = a.C + (a.core_by_q ? (long)(t % 3) * s1 * s2 * s3 : 0L);
  double* Y1 = a.ws + ((long)t * 3 + q) * ((long)r1 * s3 * (s2 + r2));
  double* Y2 = Y1 + (long)r1 * s2 * s3;
  // 2. Y1[b3][b2][a1] = sum_b1 M1[a1][b1] C[b3][b2][b1]
  for (long idx = threadIdx.x; idx < (long)s3 * s2 * r1; idx += blockDim.x) {
    const int a1 = (int)(idx % r1);
    const long bb = idx / r1;  // b3 s2 + b2
    const F* crow = Ct + bb * s1;
    double acc = 0.0;
    for (int b1 = 0; b1 < s1; ++b1) acc += M1[a1 * s1 + b1] * (double)crow[b1];
    Y1[idx] = acc;
  }
  __syncthreads();
  // 3. Y2[b3][a2][a1] = sum_b2 M2[a2][b2] Y1[b3][b2][a1]
  for (long idx = threadIdx.x; idx < (long)s3 * r2 * r1; idx += blockDim.x) {
    const int a1 = (int)(idx % r1);
    const int a2 = (int)((idx / r1) % r2);
    const long b3 = idx / ((long)r1 * r2);
    double acc = 0.0;
    for (int b2 = 0; b2 < s2; ++b2) acc += M2[a2 * s2 + b2] * Y1[(b3 * s2 + b2) * r1 + a1];
    Y2[idx] = acc;
  }
  __syncthreads();
  // 4. X = sum_a G^(q)[a3][a2][a1] sum_b3 M3[a3][b3] Y2[b3][a2][a1]
  const F* Gq = a.G + (long)q * r1 * r2 * r3;
  double x = 0.0;
  for (long idx = threadIdx.x; idx < (long)r3 * r2 * r1; idx += blockDim.x) {
    const long a21 = idx % ((long)r2 * r1);
    const int a3 = (int)(idx / ((long)r2 * r1));
    double acc = 0.0;
    for (int b3 = 0; b3 < s3; ++b3) acc += M3[a3 * s3 + b3] * Y2[(long)b3 * r2 * r1 + a21];
    x += (double)Gq[idx] * acc;
  }
  x = en_warp_sum(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < nw; ++i) v += red[i];
    a.part[(long)t * 3 + q] = (a.w ? (double)a.w[t] : 1.0) * v;
  }
}

// The same energy for a TT magnetization (Eq. tt_3d_1) and the 3M trains of its potential: one
// block per (term t, component q); the inner product of two trains contracts the first-core Gram
// M1[a1][b1], the middle-core Gram M2[(a1 a2)][(b1 b2)] and the last-core Gram M3[a2][b2]:
//   <A, B'> = sum_{a2, b2} M3[a2][b2] sum_{a1, b1} M1[a1][b1] M2[(a1 a2)][(b1 b2)],
// with D_q applied to the axis-q core of the term.
struct EnTT {
  int n[3];
  double inv2h[3];
  int r1, r2;                    // ranks of the magnetization and of every term
  const float* A[3];             // magnetization cores, component q at A[p] + q * (size of core p)
  const float* B[3];             // term cores, term t at B[p] + t * (size of core p)
  const float* w;                // term weights
  int T;
  double* part;                  // [T][3]
};

__global__ void __launch_bounds__(256) tt_energy_kernel(const __grid_constant__ EnTT a) {
  extern __shared__ double sg[];
  __shared__ double red[32];
  __shared__ float tA[64 * 33], tB[64 * 33];
  const int t = blockIdx.x, q = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int r1 = a.r1, r2 = a.r2, r12 = r1 * r2;
  const int rows[3] = {r1, r12, r2};
  double* Mg[3] = {sg, sg + r1 * r1, sg + r1 * r1 + (long)r12 * r12};
  for (int p = 0; p < 3; ++p) {
    const int n = a.n[p], rp = rows[p];
    block_gram(a.A[p] + (long)q * rp * n, rp, a.B[p] + (long)t * rp * n, rp, n, p == q, a.inv2h[p], tA, tB,
               Mg[p]);
  }
  __syncthreads();
  double x = 0.0;
  for (int e = threadIdx.x; e < r2 * r2; e += blockDim.x) {
    const int a2 = e / r2, b2 = e % r2;
    double s = 0.0;
    for (int a1 = 0; a1 < r1; ++a1)
      for (int b1 = 0; b1 < r1; ++b1) s += Mg[0][a1 * r1 + b1] * Mg[1][(long)(a1 * r2 + a2) * r12 + b1 * r2 + b2];
    x += s * Mg[2][e];
  }
  x = en_warp_sum(x);
  if (lane == 0) red[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < nw; ++i) v += red[i];
    a.part[(long)t * 3 + q] = (double)a.w[t] * v;
  }
}

// energy = scale * sum part[0..count) in a fixed order (one block)
__global__ void __launch_bounds__(256) energy_sum_kernel(long count, const double* part, double scale, double* energy) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  acc = en_warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    *energy = scale * v;
  }
}

template <typename F>
static demag_status run_tucker_energy(demag_plan* P, EnTuckerT<F>& a, double* energy, cudaStream_t st,
                                      const char* who) {
  for (int p = 0; p < 3; ++p)
    if (a.r[p] < 1 || a.r[p] > kEnMaxRank || a.s[p] < 1 || a.s[p] > kEnMaxRank)
      return set_error(P, DEMAG_EINVAL, "%s: ranks must be in [1, %d]", who, kEnMaxRank);
  for (int p = 0; p < 3; ++p) {
    a.n[p] = P->n[p];
    a.inv2h[p] = 0.5 / P->h[p];
  }
  const size_t smem = sizeof(double) * ((size_t)a.r[0] * a.s[0] + (size_t)a.r[1] * a.s[1] + (size_t)a.r[2] * a.s[2]);
  if (smem + en_static_smem<F>() > 48 * 1024) {  // dynamic plus the kernel's static tiles
    static unsigned long long done = 0;  // one per instantiation
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(done & (1ull << (dev & 63)))) {
      DEMAG_CUDA(P, cudaFuncSetAttribute(tucker_energy_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(double) * 3 * kEnMaxRank * kEnMaxRank)));
      done |= 1ull << (dev & 63);
    }
  }
  const long blocks = (long)a.T * 3;
  const long per = (long)a.r[0] * a.s[2] * (a.s[1] + a.r[1]);
  void* mem = nullptr;
  DEMAG_CUDA(P, cudaMallocAsync(&mem, sizeof(double) * (size_t)(blocks * per + blocks), st));
  a.ws = static_cast<double*>(mem);
  a.part = a.ws + blocks * per;
  DEMAG_LAUNCH(P, kFamEnergy, st, tucker_energy_kernel<F><<<dim3(a.T, 3), 256, smem, st>>>(a));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const double vol = P->h[0] * P->h[1] * P->h[2];
    DEMAG_LAUNCH(P, kFamEnergy, st, energy_sum_kernel<<<1, 256, 0, st>>>(blocks, a.part, 0.5 * vol, energy));
    e = cudaGetLastError();
  }
  cudaFreeAsync(mem, st);
  if (e != cudaSuccess) return cuda_error(P, e, who);
  return DEMAG_OK;
}

constexpr int kEnMaxTTRank = 64;  // r1 r2: the middle core's rows, at most 64 per Gram side

// The Tucker application in FP64 for the energy study after Alg. 2: with FP32 factors the
// study's energy error stops falling near 5e-7 (n >= 2048), while the method's own error keeps
// falling.  Every factor T_{k,q,p} V^(q,p) (Eq. kron_eval_tuck; T Toeplitz with
// T[i][j] = gen[i - j], E off the component's axis, F on it) is summed directly in FP64: one
// block per (column, node), the generator row and the input column in shared memory, each
// thread a set of outputs i, each sum over j in a fixed order.
struct TuckDirect {
  int n[3], r[3];
  int glen;
  const double* gen;   // [M][2][3][glen], type 0 = E, 1 = F, entry d + n_p - 1
  const double* V;     // blocks (q, p), each [r_p][n_p]
  double* out[3];      // axis p: [M][3][r_p][n_p]
};

__global__ void __launch_bounds__(256) tucker_direct_fp64_kernel(const __grid_constant__ TuckDirect a) {
  extern __shared__ double sh[];
  const int k = blockIdx.y;
  const int per_q = a.r[0] + a.r[1] + a.r[2];
  int j = blockIdx.x;
  const int q = j / per_q;
  j -= q * per_q;
  int p = 0;
  while (j >= a.r[p]) {
    j -= a.r[p];
    ++p;
  }
  const int n = a.n[p];
  const int type = p == q ? 1 : 0;
  const double* g = a.gen + (((long)k * 2 + type) * 3 + p) * a.glen;
  long voff = (long)q * ((long)a.r[0] * a.n[0] + (long)a.r[1] * a.n[1] + (long)a.r[2] * a.n[2]);
  for (int pp = 0; pp < p; ++pp) voff += (long)a.r[pp] * a.n[pp];
  const double* v = a.V + voff + (long)j * n;
  double* vs = sh;      // [n]
  double* gs = sh + n;  // [2 n - 1]
  for (int i = threadIdx.x; i < n; i += blockDim.x) vs[i] = v[i];
  for (int i = threadIdx.x; i < 2 * n - 1; i += blockDim.x) gs[i] = g[i];
  __syncthreads();
  double* out = a.out[p] + (((long)k * 3 + q) * a.r[p] + j) * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double* gi = gs + i + n - 1;  // gi[-jj] = gen[i - jj]
    double acc = 0.0;
    for (int jj = 0; jj < n; ++jj) acc = fma(gi[-jj], vs[jj], acc);
    out[i] = acc;
  }
}

// term weights of the Tucker application, w[k][q] = c s omega_k
__global__ void tucker_weights_fp64_kernel(int M, const double* scale, double* w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * M; i += gridDim.x * blockDim.x) w[i] = scale[i / 3];
}

constexpr size_t kDirectSmemMax = 200 * 1024;  // 8 (3 nmax - 1) bytes: nmax up to 8533

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_energy_tt(demag_plan* P, const int r[2], const float* G1, const float* G2,
                                        const float* G3, const float* out_w, const float* oG1, const float* oG2,
                                        const float* oG3, double* energy, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy_tt: plan is NULL");
  if (!r || !G1 || !G2 || !G3 || !out_w || !oG1 || !oG2 || !oG3 || !energy)
    return set_error(P, DEMAG_EINVAL, "demag_energy_tt: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy_tt");
  if (u != DEMAG_OK) return u;
  if (r[0] < 1 || r[1] < 1 || r[0] > kEnMaxRank || r[1] > kEnMaxRank || r[0] * r[1] > kEnMaxTTRank)
    return set_error(P, DEMAG_EINVAL, "demag_energy_tt: ranks must be in [1, %d] with r1 r2 <= %d", kEnMaxRank,
                     kEnMaxTTRank);
  cudaStream_t st = (cudaStream_t)stream;
  EnTT a{};
  for (int p = 0; p < 3; ++p) {
    a.n[p] = P->n[p];
    a.inv2h[p] = 0.5 / P->h[p];
  }
  a.r1 = r[0];
  a.r2 = r[1];
  a.A[0] = G1;
  a.A[1] = G2;
  a.A[2] = G3;
  a.B[0] = oG1;
  a.B[1] = oG2;
  a.B[2] = oG3;
  a.w = out_w;
  a.T = 3 * P->M;
  const int r12 = r[0] * r[1];
  const size_t smem = sizeof(double) * ((size_t)r[0] * r[0] + (size_t)r12 * r12 + (size_t)r[1] * r[1]);
  if (smem + kEnStaticSmem > 48 * 1024) {  // dynamic plus the kernels' static tiles
    static unsigned long long done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(done & (1ull << (dev & 63)))) {
      // largest request: r1, r2 <= 64 and r1 r2 <= 64 give at most 3 * 64^2 doubles (96 KB)
      const int cap = (int)(sizeof(double) * ((size_t)kEnMaxTTRank * kEnMaxTTRank + 2 * kEnMaxRank * kEnMaxRank));
      DEMAG_CUDA(P, cudaFuncSetAttribute(tt_energy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
      done |= 1ull << (dev & 63);
    }
  }
  const long blocks = (long)a.T * 3;
  void* mem = nullptr;
  DEMAG_CUDA(P, cudaMallocAsync(&mem, sizeof(double) * (size_t)blocks, st));
  a.part = static_cast<double*>(mem);
  DEMAG_LAUNCH(P, kFamEnergy, st, tt_energy_kernel<<<dim3(a.T, 3), 256, smem, st>>>(a));
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    const double vol = P->h[0] * P->h[1] * P->h[2];
    DEMAG_LAUNCH(P, kFamEnergy, st, energy_sum_kernel<<<1, 256, 0, st>>>(blocks, a.part, 0.5 * vol, energy));
    e = cudaGetLastError();
  }
  cudaFreeAsync(mem, st);
  if (e != cudaSuccess) return cuda_error(P, e, "demag_energy_tt");
  return DEMAG_OK;
}

extern "C" demag_status demag_energy_tucker(demag_plan* P, const int r[3], const float* core, const float* V,
                                            const float* out_w, const float* out_V, double* energy, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy_tucker: plan is NULL");
  if (!r || !core || !V || !out_w || !out_V || !energy)
    return set_error(P, DEMAG_EINVAL, "demag_energy_tucker: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy_tucker");  // uniform stencils and cell volume
  if (u != DEMAG_OK) return u;
  EnTucker a{};
  for (int p = 0; p < 3; ++p) a.r[p] = a.s[p] = r[p];
  a.G = core;
  a.V = V;
  a.C = core;
  a.core_by_q = 1;
  const long per_mode[3] = {(long)P->M * 3 * r[0] * P->n[0], (long)P->M * 3 * r[1] * P->n[1],
                            (long)P->M * 3 * r[2] * P->n[2]};
  a.W[0] = out_V;
  a.W[1] = out_V + per_mode[0];
  a.W[2] = out_V + per_mode[0] + per_mode[1];
  a.w = out_w;
  a.T = 3 * P->M;
  return run_tucker_energy(P, a, energy, (cudaStream_t)stream, "demag_energy_tucker");
}

extern "C" demag_status demag_energy_tucker_phi(demag_plan* P, const int r[3], const float* core, const float* V,
                                                const int rho[3], const float* phi_core, const float* phi_U,
                                                double* energy, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy_tucker_phi: plan is NULL");
  if (!r || !core || !V || !rho || !phi_core || !phi_U || !energy)
    return set_error(P, DEMAG_EINVAL, "demag_energy_tucker_phi: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy_tucker_phi");
  if (u != DEMAG_OK) return u;
  EnTucker a{};
  for (int p = 0; p < 3; ++p) {
    a.r[p] = r[p];
    a.s[p] = rho[p];
  }
  a.G = core;
  a.V = V;
  a.C = phi_core;
  a.core_by_q = 0;
  a.W[0] = phi_U;
  a.W[1] = phi_U + (long)rho[0] * P->n[0];
  a.W[2] = a.W[1] + (long)rho[1] * P->n[1];
  a.w = nullptr;
  a.T = 1;
  return run_tucker_energy(P, a, energy, (cudaStream_t)stream, "demag_energy_tucker_phi");
}

extern "C" demag_status demag_energy_tucker_fp64(demag_plan* P, const int r[3], const double* core, const double* V,
                                                 double* energy, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy_tucker_fp64: plan is NULL");
  if (!r || !core || !V || !energy) return set_error(P, DEMAG_EINVAL, "demag_energy_tucker_fp64: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy_tucker_fp64");
  if (u != DEMAG_OK) return u;
  for (int p = 0; p < 3; ++p)
    if (r[p] < 1 || r[p] > kEnMaxRank)
      return set_error(P, DEMAG_EINVAL, "demag_energy_tucker_fp64: ranks must be in [1, %d]", kEnMaxRank);
  const size_t smem = sizeof(double) * (3 * (size_t)P->nmax - 1);
  if (smem > kDirectSmemMax)
    return set_error(P, DEMAG_EUNSUPPORTED, "demag_energy_tucker_fp64: %d cells per axis exceed the limit of %d",
                     P->nmax, (int)((kDirectSmemMax / sizeof(double) + 1) / 3));
  cudaStream_t st = (cudaStream_t)stream;
  if (smem > 48 * 1024) {
    static unsigned long long done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(done & (1ull << (dev & 63)))) {
      DEMAG_CUDA(P, cudaFuncSetAttribute(tucker_direct_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDirectSmemMax));
      done |= 1ull << (dev & 63);
    }
  }
  const int M = P->M;
  const long per_mode[3] = {(long)M * 3 * r[0] * P->n[0], (long)M * 3 * r[1] * P->n[1],
                            (long)M * 3 * r[2] * P->n[2]};
  void* mem = nullptr;
  DEMAG_CUDA(P, cudaMallocAsync(&mem, sizeof(double) * (size_t)(per_mode[0] + per_mode[1] + per_mode[2] + 3 * M), st));
  double* outV = static_cast<double*>(mem);
  double* w = outV + per_mode[0] + per_mode[1] + per_mode[2];
  TuckDirect d{};
  for (int p = 0; p < 3; ++p) {
    d.n[p] = P->n[p];
    d.r[p] = r[p];
  }
  d.glen = P->glen;
  d.gen = P->gen64;
  d.V = V;
  d.out[0] = outV;
  d.out[1] = outV + per_mode[0];
  d.out[2] = outV + per_mode[0] + per_mode[1];
  DEMAG_LAUNCH(P, kFamEnergy, st,
               tucker_direct_fp64_kernel<<<dim3(3 * (r[0] + r[1] + r[2]), M), 256, smem, st>>>(d));
  DEMAG_LAUNCH(P, kFamEnergy, st, tucker_weights_fp64_kernel<<<1, 256, 0, st>>>(M, P->scale, w));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFreeAsync(mem, st);
    return cuda_error(P, e, "demag_energy_tucker_fp64");
  }
  EnTuckerT<double> a{};
  for (int p = 0; p < 3; ++p) a.r[p] = a.s[p] = r[p];
  a.G = core;
  a.V = V;
  a.C = core;
  a.core_by_q = 1;
  a.W[0] = d.out[0];
  a.W[1] = d.out[1];
  a.W[2] = d.out[2];
  a.w = w;
  a.T = 3 * M;
  demag_status s = run_tucker_energy(P, a, energy, st, "demag_energy_tucker_fp64");
  cudaFreeAsync(mem, st);
  return s;
}
