// Full format: the Kronecker operator by chained mode products on CUDA cores.
//
// Cor. 3 (Eq. kron_operator) with the mode product of Sec. 2.2 (Eq. modemul):
// per node k and component q the three Toeplitz factors act along i1, i2, i3.
// Per node the nine products share work (8 GEMMs of n^4 multiply-adds):
//   mode 1:  Y1 = m1 x_1 F,  Y2 = m2 x_1 E,  Y3 = m3 x_1 E
//   mode 2:  U = Y1 x_2 E + Y2 x_2 F,  V = Y3 x_2 E
//   mode 3:  phi = sum_k (U_k x_3 S_k E + V_k x_3 S_k F),  S_k = c s omega_k
// and the node sum of the last stage is one contraction of length 2 n3 M.
//
// Every stage is a "TN" GEMM whose output is stored transposed:
//   C[a][row] = alpha * sum_pairs sum_kk A[row][kk] * B[a][kk],
// A = the field with its contraction index contiguous, B = the n x n factor.
// Storing [a][row] rotates the axes (i3,i2,i1) -> (i1,i3,i2) -> (i2,i1,i3) ->
// (i3,i2,i1), so every stage reads its contraction index contiguously and the
// final stage writes phi in [i3][i2][i1] order.  The same kernel serves the
// adjoint (one field in, three out) and the FP64 form.
#include <vector>

#include "internal.h"

namespace demag {

constexpr int kMaxJobs = 64;
constexpr int kMaxPairs = 3 * kMaxTerms + 8;  // the adjoint node sum: 3 jobs of M pairs

struct GemmJob {
  int rows, ncol, K;
  int lda, ldb, ldc;
  int pair0, npairs;
  int tiles_m, tiles_n, tile0;
  float alpha;
  void* C;
};

struct GemmBatch {
  int njobs, total_tiles;
  GemmJob jobs[kMaxJobs];
  const void* A[kMaxPairs];
  const void* B[kMaxPairs];
};

template <typename T> struct SimtCfg;
template <> struct SimtCfg<float> { static constexpr int TM = 8, BK = 8; };
template <> struct SimtCfg<double> { static constexpr int TM = 4, BK = 8; };

// 256 threads as 16 x 16; each thread owns TM rows x TM columns of the tile.
template <typename T>
__global__ void __launch_bounds__(256) gemm_tn_kernel(const __grid_constant__ GemmBatch batch) {
  constexpr int TM = SimtCfg<T>::TM, BK = SimtCfg<T>::BK;
  constexpr int BM = 16 * TM, BN = 16 * TM;
  constexpr int LA = BM * BK / 256;  // elements each thread loads per operand
  __shared__ T As[2][BK][BM + 4];  // +4: conflict-free transposed stores
  __shared__ T Bs[2][BK][BN + 4];

  int tile = blockIdx.x;
  int j = 0;
  while (j + 1 < batch.njobs && tile >= batch.jobs[j + 1].tile0) ++j;
  const GemmJob& J = batch.jobs[j];
  tile -= J.tile0;
  const int tm = tile % J.tiles_m, tn = tile / J.tiles_m;
  const int row0 = tm * BM, col0 = tn * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

  T acc[TM][TM];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TM; ++b) acc[a][b] = (T)0;

  const int nk = (J.K + BK - 1) / BK;
  const int steps = nk * J.npairs;
  T ra[LA], rb[LA];

  auto load = [&](int step) {
    const int pr = J.pair0 + step / nk;
    const int k0 = (step % nk) * BK;
    const T* A = (const T*)batch.A[pr];
    const T* B = (const T*)batch.B[pr];
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      int idx = threadIdx.x + i * 256;
      int r = idx / BK, kk = idx % BK;
      int gk = k0 + kk;
      int gr = row0 + r, gc = col0 + r;
      ra[i] = (gr < J.rows && gk < J.K) ? A[(long)gr * J.lda + gk] : (T)0;
      rb[i] = (gc < J.ncol && gk < J.K) ? B[(long)gc * J.ldb + gk] : (T)0;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      int idx = threadIdx.x + i * 256;
      int r = idx / BK, kk = idx % BK;
      As[buf][kk][r] = ra[i];
      Bs[buf][kk][r] = rb[i];
    }
  };

  if (steps > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int s = 0; s < steps; ++s) {
    const int cur = s & 1;
    if (s + 1 < steps) load(s + 1);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T av[TM], bv[TM];
#pragma unroll
      for (int a = 0; a < TM / 2; ++a) {
        av[a] = As[cur][kk][tx * (TM / 2) + a];
        av[a + TM / 2] = As[cur][kk][BM / 2 + tx * (TM / 2) + a];
        bv[a] = Bs[cur][kk][ty * (TM / 2) + a];
        bv[a + TM / 2] = Bs[cur][kk][BN / 2 + ty * (TM / 2) + a];
      }
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] += av[a] * bv[b];
    }
    if (s + 1 < steps) store(cur ^ 1);
    __syncthreads();
  }

  T* C = (T*)J.C;
  const T alpha = (T)J.alpha;
#pragma unroll
  for (int b = 0; b < TM; ++b) {
    const int gc = col0 + (b < TM / 2 ? ty * (TM / 2) + b : BN / 2 + ty * (TM / 2) + b - TM / 2);
    if (gc >= J.ncol) continue;
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int gr = row0 + (a < TM / 2 ? tx * (TM / 2) + a : BM / 2 + tx * (TM / 2) + a - TM / 2);
      if (gr < J.rows) C[(long)gc * J.ldc + gr] = alpha * acc[a][b];
    }
  }
}

// ---------------------------------------------------------------- host side

class BatchBuilder {
 public:
  BatchBuilder() { b_.njobs = 0; b_.total_tiles = 0; npairs_ = 0; overflow_ = false; }
  void add(int rows, int ncol, int K, int lda, int ldb, int ldc, void* C, float alpha,
           const std::vector<std::pair<const void*, const void*>>& pairs, int bm) {
    if (b_.njobs >= kMaxJobs || npairs_ + (int)pairs.size() > kMaxPairs) {
      overflow_ = true;  // reported by launch_batch; nothing is written past the tables
      return;
    }
    GemmJob& J = b_.jobs[b_.njobs++];
    J.rows = rows; J.ncol = ncol; J.K = K;
    J.lda = lda; J.ldb = ldb; J.ldc = ldc;
    J.pair0 = npairs_;
    J.npairs = (int)pairs.size();
    for (auto& pr : pairs) {
      b_.A[npairs_] = pr.first;
      b_.B[npairs_] = pr.second;
      ++npairs_;
    }
    J.tiles_m = (rows + bm - 1) / bm;
    J.tiles_n = (ncol + bm - 1) / bm;
    J.tile0 = b_.total_tiles;
    J.alpha = alpha;
    J.C = C;
    b_.total_tiles += J.tiles_m * J.tiles_n;
  }
  const GemmBatch& get() const { return b_; }
  bool overflow() const { return overflow_; }

 private:
  GemmBatch b_;
  int npairs_;
  bool overflow_;
};

template <typename T>
static cudaError_t launch_batch(demag_plan* P, const BatchBuilder& bb, cudaStream_t st) {
  if (bb.overflow()) return cudaErrorInvalidValue;  // a job table exceeded its fixed capacity
  const GemmBatch& b = bb.get();
  if (b.total_tiles == 0) return cudaSuccess;
  DEMAG_LAUNCH(P, kFamGemmSimt, st, gemm_tn_kernel<T><<<b.total_tiles, 256, 0, st>>>(b));
  return cudaGetLastError();
}

// T[k][type][axis] blocks: n_p x n_p row-major, T[i][j] = gen[i-j+n_p-1],
// axis-3 blocks multiplied by S_k = c s omega_k.
template <typename T>
__global__ void dense_factor_kernel(int M, int glen, int n0, int n1, int n2, size_t tgroup, size_t off1,
                                    size_t off2, const double* gen, const double* scale, T* out,
                                    const double* fac = nullptr, bool transpose = false) {
  const size_t total = (size_t)M * 2 * tgroup;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    size_t e = idx % tgroup;
    size_t kt = idx / tgroup;  // k*2 + type
    int axis, n;
    size_t local;
    if (e < off1) { axis = 0; n = n0; local = e; }
    else if (e < off2) { axis = 1; n = n1; local = e - off1; }
    else { axis = 2; n = n2; local = e - off2; }
    int i = (int)(local / n), jj = (int)(local % n);
    if (transpose) {
      const int t = i;
      i = jj;
      jj = t;
    }
    // Toeplitz generator (uniform grid) or the full matrix (non-uniform grid)
    double v = fac ? fac[kt * tgroup + (e - local) + (size_t)i * n + jj] : gen[(kt * 3 + axis) * glen + (i - jj + n - 1)];
    if (axis == 2) v *= scale[kt / 2];
    out[idx] = (T)v;
  }
}

template <typename T>
static const T* factor(const demag_plan* P, const T* base, int k, int type, int axis) {
  return base + ((size_t)k * 2 + type) * P->tgroup + P->toff[axis];
}

demag_status ensure_dense_factors(demag_plan* P, demag_precision prec, cudaStream_t st) {
  const size_t total = (size_t)P->M * 2 * P->tgroup;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (prec == DEMAG_FP64) {
    if (P->T64) return DEMAG_OK;
    DEMAG_CUDA(P, cudaMalloc(&P->T64, sizeof(double) * total));
    DEMAG_LAUNCH(P, kFamSetup, st,
                 dense_factor_kernel<double><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                     P->tgroup, P->toff[1], P->toff[2], P->gen64,
                                                                     P->scale, P->T64, P->fac64));
  } else {
    if (P->T32) return DEMAG_OK;
    DEMAG_CUDA(P, cudaMalloc(&P->T32, sizeof(float) * total));
    DEMAG_LAUNCH(P, kFamSetup, st,
                 dense_factor_kernel<float><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                    P->tgroup, P->toff[1], P->toff[2], P->gen64,
                                                                    P->scale, P->T32, P->fac64));
  }
  DEMAG_LAUNCHED(P, "dense_factor_kernel");
  return DEMAG_OK;
}

// Transposed factor tables of a non-uniform plan, for the adjoint on CUDA
// cores: (P^(q))^T = c sum_k omega_k U3^T (x) U2^T (x) U1^T.
static demag_status ensure_transposed_factors(demag_plan* P, demag_precision prec, cudaStream_t st) {
  const size_t total = (size_t)P->M * 2 * P->tgroup;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (prec == DEMAG_FP64) {
    if (P->T64t) return DEMAG_OK;
    DEMAG_CUDA(P, cudaMalloc(&P->T64t, sizeof(double) * total));
    DEMAG_LAUNCH(P, kFamSetup, st,
                 dense_factor_kernel<double><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                     P->tgroup, P->toff[1], P->toff[2], P->gen64,
                                                                     P->scale, P->T64t, P->fac64, true));
  } else {
    if (P->T32t) return DEMAG_OK;
    DEMAG_CUDA(P, cudaMalloc(&P->T32t, sizeof(float) * total));
    DEMAG_LAUNCH(P, kFamSetup, st,
                 dense_factor_kernel<float><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                    P->tgroup, P->toff[1], P->toff[2], P->gen64,
                                                                    P->scale, P->T32t, P->fac64, true));
  }
  DEMAG_LAUNCHED(P, "dense_factor_kernel (transposed)");
  return DEMAG_OK;
}

size_t workspace_bytes(const demag_plan* P, demag_precision prec) {
  const size_t N = field_size(P);
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) return tc_workspace_bytes(P, prec);
  // forward: Y (3 fields) + U,V per node; adjoint: Y (2) + 3 per node.
  // FP64 also keeps double copies of the input and output fields (3 + 3).
  size_t fields = 3 * (size_t)P->M + 3;
  if (prec == DEMAG_FP64) fields += 6;
  return fields * N * (prec == DEMAG_FP64 ? sizeof(double) : sizeof(float));
}

demag_status ensure_workspace(demag_plan* P, demag_precision prec) {
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) return tc_prepare(P, prec, 0);  // owns its buffers
  demag::Workspace& w = P->ws[prec];
  const size_t need = workspace_bytes(P, prec);
  if (w.base && w.bytes >= need) return DEMAG_OK;
  if (w.base) cudaFree(w.base);
  w.base = nullptr;
  w.bytes = 0;
  cudaError_t e = cudaMalloc(&w.base, need);
  if (e != cudaSuccess) return cuda_error(P, e, "workspace allocation");
  w.bytes = need;
  return DEMAG_OK;
}

template <typename T>
__global__ void convert_kernel(const float* in, T* out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (T)in[i];
}
__global__ void narrow_kernel(const double* in, float* out, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// forward: m (3 fields, type T) -> phi (type T) using workspace `ws` of type T
template <typename T>
// Tax[p]: the factor table used along axis p (the analytic stray field swaps
// in the derivative factors along one axis); alpha scales the result.
static demag_status simt_forward(demag_plan* P, const T* m, T* phi, const T* const (&Tax)[3], T* ws,
                                 cudaStream_t st, float alpha = 1.f) {
  constexpr int BM = 16 * SimtCfg<T>::TM;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const size_t N = field_size(P);
  T* Y = ws;                 // 3 fields
  T* UV = ws + 3 * N;        // [M][2] fields
  const int M = P->M;
  for (int k = 0; k < M; ++k) {
    BatchBuilder b1;
    for (int q = 0; q < 3; ++q) {
      const T* B = factor(P, Tax[0], k, q == 0 ? 1 : 0, 0);
      b1.add(n3 * n2, n1, n1, n1, n1, n3 * n2, Y + q * N, 1.f, {{m + q * N, B}}, BM);
    }
    cudaError_t e = launch_batch<T>(P, b1, st);
    if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (mode 1)");
    BatchBuilder b2;
    const T* E2 = factor(P, Tax[1], k, 0, 1);
    const T* F2 = factor(P, Tax[1], k, 1, 1);
    b2.add(n1 * n3, n2, n2, n2, n2, n1 * n3, UV + (2 * k) * N, 1.f, {{Y, E2}, {Y + N, F2}}, BM);
    b2.add(n1 * n3, n2, n2, n2, n2, n1 * n3, UV + (2 * k + 1) * N, 1.f, {{Y + 2 * N, E2}}, BM);
    e = launch_batch<T>(P, b2, st);
    if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (mode 2)");
  }
  BatchBuilder b3;
  std::vector<std::pair<const void*, const void*>> pairs;
  for (int k = 0; k < M; ++k) {
    pairs.push_back({UV + (2 * k) * N, factor(P, Tax[2], k, 0, 2)});
    pairs.push_back({UV + (2 * k + 1) * N, factor(P, Tax[2], k, 1, 2)});
  }
  b3.add(n2 * n1, n3, n3, n3, n3, n2 * n1, phi, alpha, pairs, BM);
  cudaError_t e = launch_batch<T>(P, b3, st);
  if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (mode 3)");
  return DEMAG_OK;
}

// adjoint: y (1 field) -> g (3 fields).  Uniform grid: g^(q) = -P^(q) y with
// the forward tables (sign -1); non-uniform grid: the transposed tables and
// sign +1.
template <typename T>
static demag_status simt_adjoint(demag_plan* P, const T* y, T* g, const T* Tm, T* ws, cudaStream_t st,
                                 float sign = -1.f) {
  constexpr int BM = 16 * SimtCfg<T>::TM;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const size_t N = field_size(P);
  T* Y = ws;            // 2 fields: F1 y, E1 y
  T* Z = ws + 2 * N;    // [M][3]
  const int M = P->M;
  for (int k = 0; k < M; ++k) {
    BatchBuilder b1;
    b1.add(n3 * n2, n1, n1, n1, n1, n3 * n2, Y, 1.f, {{y, factor(P, Tm, k, 1, 0)}}, BM);
    b1.add(n3 * n2, n1, n1, n1, n1, n3 * n2, Y + N, 1.f, {{y, factor(P, Tm, k, 0, 0)}}, BM);
    cudaError_t e = launch_batch<T>(P, b1, st);
    if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (adjoint mode 1)");
    BatchBuilder b2;
    const T* E2 = factor(P, Tm, k, 0, 1);
    const T* F2 = factor(P, Tm, k, 1, 1);
    b2.add(n1 * n3, n2, n2, n2, n2, n1 * n3, Z + (3 * k) * N, 1.f, {{Y, E2}}, BM);
    b2.add(n1 * n3, n2, n2, n2, n2, n1 * n3, Z + (3 * k + 1) * N, 1.f, {{Y + N, F2}}, BM);
    b2.add(n1 * n3, n2, n2, n2, n2, n1 * n3, Z + (3 * k + 2) * N, 1.f, {{Y + N, E2}}, BM);
    e = launch_batch<T>(P, b2, st);
    if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (adjoint mode 2)");
  }
  BatchBuilder b3;
  for (int q = 0; q < 3; ++q) {
    std::vector<std::pair<const void*, const void*>> pairs;
    for (int k = 0; k < M; ++k) pairs.push_back({Z + (3 * k + q) * N, factor(P, Tm, k, q == 2 ? 1 : 0, 2)});
    b3.add(n2 * n1, n3, n3, n3, n3, n2 * n1, g + q * N, sign, pairs, BM);
  }
  cudaError_t e = launch_batch<T>(P, b3, st);
  if (e != cudaSuccess) return cuda_error(P, e, "gemm_tn_kernel (adjoint mode 3)");
  return DEMAG_OK;
}

static int conv_blocks(size_t count) {
  size_t b = (count + 255) / 256;
  return (int)(b > 152 * 32 ? 152 * 32 : b);
}

demag_status full_forward(demag_plan* P, const float* m, float* phi, demag_precision prec, cudaStream_t st) {
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) return tc_forward(P, m, phi, prec, st);
  demag_status s = ensure_dense_factors(P, prec, st);
  if (s != DEMAG_OK) return s;
  s = ensure_workspace(P, prec);
  if (s != DEMAG_OK) return s;
  const size_t N = field_size(P);
  if (prec == DEMAG_FP32) {
    const float* const tax[3] = {P->T32, P->T32, P->T32};
    return simt_forward<float>(P, m, phi, tax, (float*)P->ws[prec].base, st);
  }
  double* ws = (double*)P->ws[prec].base;
  double* m64 = ws + (3 * (size_t)P->M + 3) * N;
  double* phi64 = m64 + 3 * N;
  DEMAG_LAUNCH(P, kFamSplit, st, convert_kernel<double><<<conv_blocks(3 * N), 256, 0, st>>>(m, m64, 3 * N));
  DEMAG_LAUNCHED(P, "convert_kernel");
  const double* const tax[3] = {P->T64, P->T64, P->T64};
  s = simt_forward<double>(P, m64, phi64, tax, ws, st);
  if (s != DEMAG_OK) return s;
  DEMAG_LAUNCH(P, kFamSplit, st, narrow_kernel<<<conv_blocks(N), 256, 0, st>>>(phi64, phi, N));
  DEMAG_LAUNCHED(P, "narrow_kernel");
  return DEMAG_OK;
}

// ---------------------------------------------------------------- analytic stray field (CUDA cores)

// h_d[p] = -dphi/dxi_p for p = 1..3: the forward chain with the axis-p factor
// table replaced by the derivative table (built from the derivative generators).
demag_status simt_field(demag_plan* P, const float* m, float* hd, demag_precision prec, cudaStream_t st) {
  demag_status s = ensure_dense_factors(P, prec, st);
  if (s == DEMAG_OK) s = ensure_workspace(P, prec);
  if (s == DEMAG_OK) s = ensure_field_generators(P, st);
  if (s != DEMAG_OK) return s;
  const size_t total = (size_t)P->M * 2 * P->tgroup;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 64) blocks = 152 * 64;
  const size_t N = field_size(P);
  if (prec == DEMAG_FP32) {
    if (!P->T32d) {
      DEMAG_CUDA(P, cudaMalloc(&P->T32d, sizeof(float) * total));
      DEMAG_LAUNCH(P, kFamSetup, st,
                   dense_factor_kernel<float><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                      P->tgroup, P->toff[1], P->toff[2], P->gend,
                                                                      P->scale, P->T32d));
      DEMAG_LAUNCHED(P, "dense_factor_kernel");
    }
    for (int p = 0; p < 3 && s == DEMAG_OK; ++p) {
      const float* const tax[3] = {p == 0 ? P->T32d : P->T32, p == 1 ? P->T32d : P->T32, p == 2 ? P->T32d : P->T32};
      s = simt_forward<float>(P, m, hd + p * N, tax, (float*)P->ws[prec].base, st, -1.f);
    }
    return s;
  }
  if (!P->T64d) {
    DEMAG_CUDA(P, cudaMalloc(&P->T64d, sizeof(double) * total));
    DEMAG_LAUNCH(P, kFamSetup, st,
                 dense_factor_kernel<double><<<blocks, 256, 0, st>>>(P->M, P->glen, P->n[0], P->n[1], P->n[2],
                                                                     P->tgroup, P->toff[1], P->toff[2], P->gend,
                                                                     P->scale, P->T64d));
    DEMAG_LAUNCHED(P, "dense_factor_kernel");
  }
  double* ws = (double*)P->ws[prec].base;
  double* m64 = ws + (3 * (size_t)P->M + 3) * N;
  double* out64 = m64 + 3 * N;
  DEMAG_LAUNCH(P, kFamSplit, st, convert_kernel<double><<<conv_blocks(3 * N), 256, 0, st>>>(m, m64, 3 * N));
  DEMAG_LAUNCHED(P, "convert_kernel");
  for (int p = 0; p < 3 && s == DEMAG_OK; ++p) {
    const double* const tax[3] = {p == 0 ? P->T64d : P->T64, p == 1 ? P->T64d : P->T64, p == 2 ? P->T64d : P->T64};
    s = simt_forward<double>(P, m64, out64, tax, ws, st, -1.f);
    if (s != DEMAG_OK) break;
    DEMAG_LAUNCH(P, kFamSplit, st, narrow_kernel<<<conv_blocks(N), 256, 0, st>>>(out64, hd + p * N, N));
    DEMAG_LAUNCHED(P, "narrow_kernel");
  }
  return s;
}

demag_status full_adjoint(demag_plan* P, const float* y, float* g, demag_precision prec, cudaStream_t st) {
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) {
    // the split-precision adjoint programs rely on P^T = -P (uniform grids)
    demag_status u = require_uniform(P, "demag_apply_adjoint in split precision");
    if (u != DEMAG_OK) return u;
    return tc_adjoint(P, y, g, prec, st);
  }
  demag_status s = P->nonuniform ? ensure_transposed_factors(P, prec, st) : ensure_dense_factors(P, prec, st);
  if (s != DEMAG_OK) return s;
  s = ensure_workspace(P, prec);
  if (s != DEMAG_OK) return s;
  const size_t N = field_size(P);
  const float sign = P->nonuniform ? 1.f : -1.f;
  if (prec == DEMAG_FP32)
    return simt_adjoint<float>(P, y, g, P->nonuniform ? P->T32t : P->T32, (float*)P->ws[prec].base, st, sign);
  double* ws = (double*)P->ws[prec].base;
  double* y64 = ws + (3 * (size_t)P->M + 3) * N;
  double* g64 = y64 + 3 * N;
  DEMAG_LAUNCH(P, kFamSplit, st, convert_kernel<double><<<conv_blocks(N), 256, 0, st>>>(y, y64, N));
  DEMAG_LAUNCHED(P, "convert_kernel");
  s = simt_adjoint<double>(P, y64, g64, P->nonuniform ? P->T64t : P->T64, ws, st, sign);
  if (s != DEMAG_OK) return s;
  DEMAG_LAUNCH(P, kFamSplit, st, narrow_kernel<<<conv_blocks(3 * N), 256, 0, st>>>(g64, g, 3 * N));
  DEMAG_LAUNCHED(P, "narrow_kernel");
  return DEMAG_OK;
}

static demag_status check_prec(demag_plan* P, demag_precision prec, const char* what) {
  if ((int)prec < 0 || (int)prec > 3) return set_error(P, DEMAG_EINVAL, "%s: unknown precision %d", what, (int)prec);
  return DEMAG_OK;
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_reserve_workspace(demag_plan* P, demag_precision prec) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_reserve_workspace: plan is NULL");
  demag_status s = check_prec(P, prec, "demag_reserve_workspace");
  if (s != DEMAG_OK) return s;
  if (prec != DEMAG_TF32X3 && prec != DEMAG_BF16X3) {
    s = ensure_dense_factors(P, prec, 0);
    if (s != DEMAG_OK) return s;
  }
  s = ensure_workspace(P, prec);
  if (s != DEMAG_OK) return s;
  DEMAG_CUDA(P, cudaDeviceSynchronize());
  return DEMAG_OK;
}

extern "C" demag_status demag_apply_full(demag_plan* P, const float* m, float* phi, demag_precision prec,
                                         void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_apply_full: plan is NULL");
  demag_status s = check_prec(P, prec, "demag_apply_full");
  if (s != DEMAG_OK) return s;
  if (!m || !phi) return set_error(P, DEMAG_EINVAL, "demag_apply_full: NULL pointer");
  return full_forward(P, m, phi, prec, (cudaStream_t)stream);
}

extern "C" demag_status demag_apply_adjoint(demag_plan* P, const float* y, float* g, demag_precision prec,
                                            void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_apply_adjoint: plan is NULL");
  demag_status s = check_prec(P, prec, "demag_apply_adjoint");
  if (s != DEMAG_OK) return s;
  if (!y || !g) return set_error(P, DEMAG_EINVAL, "demag_apply_adjoint: NULL pointer");
  return full_adjoint(P, y, g, prec, (cudaStream_t)stream);
}

static demag_status check_batch(demag_plan* const* plans, const float* const* m, float* const* phi, int count,
                                demag_precision prec, const char* what) {
  if (count < 0 || (count > 0 && (!plans || !m || !phi)))
    return set_error(nullptr, DEMAG_EINVAL, "%s: bad arguments", what);
  if ((int)prec < 0 || (int)prec > (int)DEMAG_BF16X3)
    return set_error(nullptr, DEMAG_EINVAL, "%s: unknown precision %d", what, (int)prec);
  for (int i = 0; i < count; ++i) {
    if (!plans[i] || !m[i] || !phi[i]) return set_error(nullptr, DEMAG_EINVAL, "%s: NULL entry %d", what, i);
    const bool tc = prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3;
    if (tc ? !tc_ready(plans[i], prec) : !plans[i]->ws[prec].base)
      return set_error(plans[i], DEMAG_EINVAL, "%s: plan %d has no workspace", what, i);
  }
  return DEMAG_OK;
}

extern "C" demag_status demag_apply_full_batched(demag_plan* const* plans, const float* const* m,
                                                 float* const* phi, int count, demag_precision prec,
                                                 void* stream) {
  demag_status cs = check_batch(plans, m, phi, count, prec, "demag_apply_full_batched");
  if (cs != DEMAG_OK) return cs;
  if (prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3) {
    // each stage of a run of distinct plans is one grouped persistent launch;
    // a plan that repeats (it owns one set of intermediates) starts a new run
    int first = 0;
    for (int i = 1; i <= count; ++i) {
      bool repeat = false;
      for (int j = first; j < i && i < count; ++j) repeat = repeat || plans[j] == plans[i];
      if (i == count || repeat) {
        demag_status s = tc_forward_batched(plans + first, m + first, phi + first, i - first, prec,
                                            (cudaStream_t)stream);
        if (s != DEMAG_OK) return s;
        first = i;
      }
    }
    return DEMAG_OK;
  }
  for (int i = 0; i < count; ++i) {
    demag_status s = full_forward(plans[i], m[i], phi[i], prec, (cudaStream_t)stream);
    if (s != DEMAG_OK) return s;
  }
  return DEMAG_OK;
}

// ---------------------------------------------------------------- CUDA-graph form of the batched apply

struct demag_graph {
  std::vector<demag_plan*> plans;
  demag::TcBatch* batch = nullptr;  // grouped descriptors owned by this graph (tensor-core forms)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

extern "C" void demag_graph_destroy(demag_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  tc_batch_destroy(g->batch);
  delete g;
}

extern "C" demag_status demag_graph_create_batched(demag_plan* const* plans, const float* const* m,
                                                   float* const* phi, int count, demag_precision prec,
                                                   demag_graph** out) {
  if (!out) return set_error(nullptr, DEMAG_EINVAL, "demag_graph_create_batched: out is NULL");
  *out = nullptr;
  demag_status s = check_batch(plans, m, phi, count, prec, "demag_graph_create_batched");
  if (s != DEMAG_OK) return s;
  if (count == 0) return set_error(nullptr, DEMAG_EINVAL, "demag_graph_create_batched: empty batch");
  for (int i = 0; i < count; ++i)
    for (int j = 0; j < i; ++j)
      if (plans[i] == plans[j])
        return set_error(plans[i], DEMAG_EINVAL, "demag_graph_create_batched: plan %d repeats plan %d", i, j);
  const bool tc = prec == DEMAG_TF32X3 || prec == DEMAG_BF16X3;
  demag_graph* g = new demag_graph();
  g->plans.assign(plans, plans + count);
  if (tc) {
    s = tc_batch_create(plans, count, prec, &g->batch);
    if (s != DEMAG_OK) {
      demag_graph_destroy(g);
      return s;
    }
  }
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    demag_graph_destroy(g);
    return cuda_error(plans[0], e, "demag_graph_create_batched: stream");
  }
  // event timing would record into the graph: off while capturing
  std::vector<char> prof(count);
  std::vector<unsigned long long> before(count);
  for (int i = 0; i < count; ++i) {
    prof[i] = plans[i]->prof_on;
    plans[i]->prof_on = false;
    before[i] = plans[i]->launches;
  }
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (tc) {
      s = tc_batch_run(g->batch, m, phi, cs);
    } else {
      for (int i = 0; i < count && s == DEMAG_OK; ++i) s = full_forward(plans[i], m[i], phi[i], prec, cs);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    g->graph = graph;
    if (s == DEMAG_OK && e2 != cudaSuccess) s = cuda_error(plans[0], e2, "demag_graph_create_batched: capture");
  } else {
    s = cuda_error(plans[0], e, "demag_graph_create_batched: begin capture");
  }
  // the capture launched nothing: move the recorded kernels out of the counters
  unsigned long long recorded = 0;
  for (int i = 0; i < count; ++i) {
    plans[i]->prof_on = prof[i];
    recorded += plans[i]->launches - before[i];
    plans[i]->launches = before[i];
  }
  g->kernels = (int)recorded;
  cudaStreamDestroy(cs);
  if (s == DEMAG_OK && g->graph) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) s = cuda_error(plans[0], e, "demag_graph_create_batched: instantiate");
  }
  if (s != DEMAG_OK) {
    demag_graph_destroy(g);
    return s;
  }
  *out = g;
  return DEMAG_OK;
}

extern "C" demag_status demag_graph_launch(demag_graph* g, void* stream) {
  if (!g || !g->exec) return set_error(nullptr, DEMAG_EINVAL, "demag_graph_launch: graph is NULL");
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_error(g->plans[0], e, "demag_graph_launch");
  g->plans[0]->launches += (unsigned long long)g->kernels;
  return DEMAG_OK;
}

extern "C" int demag_graph_kernel_count(const demag_graph* g) { return g ? g->kernels : 0; }

// ---------------------------------------------------------------- allocation-free entry point
//
// demag_apply_full_noalloc serves callers that must not allocate device
// memory themselves or through this library: code that runs while a device
// memory pool owned by a host framework has reserved the GPU (a cudaMalloc
// from a library would fail or fragment it), latency-critical loops where
// an allocation would implicitly synchronise the device, and embedders whose
// plugin rules forbid allocation.  Everything this call needs beyond the
// caller's input and output (nodes, generators, dense factors and the
// intermediates of the mode-product chain) lives in one file-scope device
// array of fixed size, which every GPU that loads the library keeps until
// the process exits.  The arithmetic is that of demag_apply_full with
// DEMAG_FP32 (same kernels, same order).

#include <cmath>
#include <mutex>

namespace demag {

constexpr size_t kNoAllocBytes = size_t(32) << 20;  // 32 MiB of device scratch
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static void* g_noalloc_addr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of the scratch array on the current device.  Host code sees
// only a host-side stand-in for `g_noalloc_scratch`, so the address is asked
// from the runtime once per device (with that device current) and cached.
static demag_status noalloc_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(nullptr, e, "demag_apply_full_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return set_error(nullptr, DEMAG_EUNSUPPORTED, "demag_apply_full_noalloc: device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(nullptr, e, "demag_apply_full_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return DEMAG_OK;
}

static size_t na_align(size_t b) { return (b + 255) & ~size_t(255); }

// Append one job to a GEMM batch without any host heap use.
static void na_add(GemmBatch& b, int& npairs, int rows, int ncol, int K, int ldc, void* C,
                   const void* const* A, const void* const* B, int np) {
  GemmJob& J = b.jobs[b.njobs++];
  J.rows = rows; J.ncol = ncol; J.K = K;
  J.lda = K; J.ldb = K; J.ldc = ldc;
  J.pair0 = npairs;
  J.npairs = np;
  for (int i = 0; i < np; ++i) {
    b.A[npairs] = A[i];
    b.B[npairs] = B[i];
    ++npairs;
  }
  const int bm = 16 * SimtCfg<float>::TM;
  J.tiles_m = (rows + bm - 1) / bm;
  J.tiles_n = (ncol + bm - 1) / bm;
  J.tile0 = b.total_tiles;
  J.alpha = 1.f;
  J.C = C;
  b.total_tiles += J.tiles_m * J.tiles_n;
}

static demag_status na_launch(demag_plan* P, const GemmBatch& b, cudaStream_t st) {
  DEMAG_LAUNCH(P, kFamGemmSimt, st, gemm_tn_kernel<float><<<b.total_tiles, 256, 0, st>>>(b));
  DEMAG_LAUNCHED(P, "gemm_tn_kernel (allocation-free)");
  return DEMAG_OK;
}

}  // namespace demag

extern "C" demag_status demag_apply_full_noalloc(const demag_grid_desc* d, const float* m, float* phi,
                                                 void* stream) {
  using namespace demag;
  if (!d || !m || !phi) return set_error(nullptr, DEMAG_EINVAL, "demag_apply_full_noalloc: NULL pointer");
  for (int p = 0; p < 3; ++p) {
    if (d->n[p] < 1) return set_error(nullptr, DEMAG_EINVAL, "n[%d] = %d must be >= 1", p, d->n[p]);
    if (!(d->h[p] > 0.0) || !std::isfinite(d->h[p]))
      return set_error(nullptr, DEMAG_EINVAL, "h[%d] must be positive and finite", p);
  }
  if (d->R < 5 || d->R % 2 == 0)
    return set_error(nullptr, DEMAG_EINVAL, "R = %d must be odd and >= 5 (R = 2M+1)", d->R);
  if ((d->R - 1) / 2 > kMaxTerms)
    return set_error(nullptr, DEMAG_EUNSUPPORTED, "R = %d exceeds 2*%d+1", d->R, kMaxTerms);
  if (!(d->c0 > 0.0) || !std::isfinite(d->c0))
    return set_error(nullptr, DEMAG_EINVAL, "c0 must be positive and finite");

  // the fields of a plan this call needs, kept on the host stack
  demag_plan P;
  snprintf(P.err, sizeof(P.err), "no error");
  P.R = d->R;
  P.M = (d->R - 1) / 2;
  P.c0 = d->c0;
  P.s = 0.0;
  P.nmax = 0;
  for (int p = 0; p < 3; ++p) {
    P.n[p] = d->n[p];
    P.h[p] = d->h[p];
    P.s = fmax(P.s, (double)d->n[p] * d->h[p]);
    P.nmax = d->n[p] > P.nmax ? d->n[p] : P.nmax;
  }
  P.tgroup = 0;
  for (int p = 0; p < 3; ++p) {
    P.hh[p] = P.h[p] / P.s;
    P.toff[p] = P.tgroup;
    P.tgroup += (size_t)P.n[p] * P.n[p];
  }
  P.glen = 2 * P.nmax - 1;
  const int M = P.M;
  const size_t N = (size_t)P.n[0] * P.n[1] * P.n[2];

  // scratch layout: nodes [3][M], scale [M], generators [M][2][3][glen] (FP64),
  // dense factors [M][2][sum n_p^2] and the chain's fields Y (3) + U, V (2M) (FP32)
  const size_t b_nodes = na_align(sizeof(double) * 3 * M);
  const size_t b_scale = na_align(sizeof(double) * M);
  const size_t b_gen = na_align(sizeof(double) * (size_t)M * 6 * P.glen);
  const size_t b_fac = na_align(sizeof(float) * (size_t)M * 2 * P.tgroup);
  const size_t b_ws = na_align(sizeof(float) * (2 * (size_t)M + 3) * N);
  const size_t need = b_nodes + b_scale + b_gen + b_fac + b_ws;
  if (need > kNoAllocBytes)
    return set_error(nullptr, DEMAG_EUNSUPPORTED,
                     "demag_apply_full_noalloc: this grid needs %zu bytes of scratch, the fixed maximum is %zu "
                     "bytes (%d MiB); use demag_apply_full",
                     need, kNoAllocBytes, (int)(kNoAllocBytes >> 20));

  void* base = nullptr;
  demag_status s = noalloc_address(&base);
  if (s != DEMAG_OK) return s;
  unsigned char* at = static_cast<unsigned char*>(base);
  P.nodes = reinterpret_cast<double*>(at);
  P.scale = reinterpret_cast<double*>(at + b_nodes);
  P.gen64 = reinterpret_cast<double*>(at + b_nodes + b_scale);
  float* T = reinterpret_cast<float*>(at + b_nodes + b_scale + b_gen);
  float* Y = reinterpret_cast<float*>(at + b_nodes + b_scale + b_gen + b_fac);
  float* UV = Y + 3 * N;
  cudaStream_t st = (cudaStream_t)stream;

  // setup: every scratch region below is fully written before it is read,
  // so nothing has to be cleared between calls
  DEMAG_LAUNCH(&P, kFamSetup, st, nodes_kernel<<<(M + 63) / 64, 64, 0, st>>>(M, P.c0, kCPot * P.s, P.nodes, P.scale));
  DEMAG_LAUNCHED(&P, "nodes_kernel (allocation-free)");
  GridInfo g;
  for (int p = 0; p < 3; ++p) {
    g.n[p] = P.n[p];
    g.hh[p] = P.hh[p];
  }
  {
    long total = (long)M * 6 * P.glen;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    DEMAG_LAUNCH(&P, kFamSetup, st, generators_kernel<<<blocks, 256, 0, st>>>(M, P.glen, g, P.nodes, P.gen64));
    DEMAG_LAUNCHED(&P, "generators_kernel (allocation-free)");
  }
  {
    const size_t total = (size_t)M * 2 * P.tgroup;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 64) blocks = 152 * 64;
    DEMAG_LAUNCH(&P, kFamSetup, st,
                 dense_factor_kernel<float><<<blocks, 256, 0, st>>>(M, P.glen, P.n[0], P.n[1], P.n[2], P.tgroup,
                                                                    P.toff[1], P.toff[2], P.gen64, P.scale, T));
    DEMAG_LAUNCHED(&P, "dense_factor_kernel (allocation-free)");
  }

  // the mode-product chain of demag_apply_full (DEMAG_FP32)
  const int n1 = P.n[0], n2 = P.n[1], n3 = P.n[2];
  for (int k = 0; k < M; ++k) {
    GemmBatch b1;
    b1.njobs = 0;
    b1.total_tiles = 0;
    int np = 0;
    for (int q = 0; q < 3; ++q) {
      const void* A[1] = {m + q * N};
      const void* B[1] = {factor(&P, (const float*)T, k, q == 0 ? 1 : 0, 0)};
      na_add(b1, np, n3 * n2, n1, n1, n3 * n2, Y + q * N, A, B, 1);
    }
    s = na_launch(&P, b1, st);
    if (s != DEMAG_OK) return s;
    GemmBatch b2;
    b2.njobs = 0;
    b2.total_tiles = 0;
    np = 0;
    const float* E2 = factor(&P, (const float*)T, k, 0, 1);
    const float* F2 = factor(&P, (const float*)T, k, 1, 1);
    {
      const void* A[2] = {Y, Y + N};
      const void* B[2] = {E2, F2};
      na_add(b2, np, n1 * n3, n2, n2, n1 * n3, UV + (2 * k) * N, A, B, 2);
    }
    {
      const void* A[1] = {Y + 2 * N};
      const void* B[1] = {E2};
      na_add(b2, np, n1 * n3, n2, n2, n1 * n3, UV + (2 * k + 1) * N, A, B, 1);
    }
    s = na_launch(&P, b2, st);
    if (s != DEMAG_OK) return s;
  }
  GemmBatch b3;
  b3.njobs = 0;
  b3.total_tiles = 0;
  int np = 0;
  const void* A3[2 * kMaxTerms];
  const void* B3[2 * kMaxTerms];
  for (int k = 0; k < M; ++k) {
    A3[2 * k] = UV + (2 * k) * N;
    B3[2 * k] = factor(&P, (const float*)T, k, 0, 2);
    A3[2 * k + 1] = UV + (2 * k + 1) * N;
    B3[2 * k + 1] = factor(&P, (const float*)T, k, 1, 2);
  }
  na_add(b3, np, n2 * n1, n3, n3, n2 * n1, phi, A3, B3, 2 * M);
  return na_launch(&P, b3, st);
}
