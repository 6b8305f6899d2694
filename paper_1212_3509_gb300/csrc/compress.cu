// Alg. 2 with compressed kernels: Tucker compression of the CP convolution
// kernels by HOOI (Alg. 1) and their application to Tucker magnetizations.
//
// Kernel of component q (Eq. conv_pot): K^(q) = sum_k lam_k a_{1k} (x) a_{2k} (x) a_{3k},
// lam_k = c s omega_k, a_{pk} the generator F_k^(p) (p == q) or E_k^(p) (p != q),
// 2 n_p - 1 entries.  With A_p = Q_p R_p (QR of the M generator columns of one
// type and axis) every Gram matrix of an unfolding of K^(q), after projecting
// the other modes on V_s, V_r, is
//   Y_(p) Y_(p)^T = Q_p S_p Q_p^T,  S_p = R_p Lam ((B_s^T B_s) o (B_r^T B_r)) Lam R_p^T,
//   B_x = V_x^T R_x  (B_x = R_x for the HOSVD start),
// so HOSVD and the HOOI sweeps of Alg. 1 only need eigen-decompositions of
// M x M matrices: the mode-p factor is U_p = Q_p V_p, V_p the leading
// eigenvectors of S_p, and the core is C = sum_k lam_k b_{1k} (x) b_{2k} (x) b_{3k}
// with b_{pk} = V_p^T R_p[:, k].  The ranks follow the HOSVD rule of Alg. 1
// (discarded singular values of each unfolding below tol/sqrt(3) of its
// norm), the largest over the three components, so all components share one
// rank per mode; HOOI then sweeps at those ranks.  The columns of U_p are
// generators of Toeplitz matrices again (linear combinations of E or F
// generators), so the compressed kernel is applied with the circulant FFT
// kernel of the structured formats, one symbol set per component.
//
// Application (Lemma DFT_tucker, App. B Eq. t_had2): for a Tucker
// magnetization [[G^(q); V^(q,1), V^(q,2), V^(q,3)]] the result is
//   sum_q [[C^(q) (x) G^(q); W^(q,1), W^(q,2), W^(q,3)]],  W^(q,p)[:, (i, l)] = T(U_p^(q)[:, i]) V^(q,p)[:, l],
// factors written [rho_p][3][r_p][n_p] (i major) and cores
// [(rho3 r3)][(rho2 r2)][(rho1 r1)] with the same (i, l) index order.
// Setup arithmetic is FP64; the application is FP32 (like the uncompressed
// structured path).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

namespace demag {

struct Compressed {
  double tol = 0.0;
  int rho[3] = {0, 0, 0};
  double* cgen = nullptr;   // [rhomax][3 q][3 p][glen] compressed generators
  float* csym = nullptr;    // [rhomax][3][3][Lmax/2 + 1]
  float2* cpair = nullptr;  // [rhomax][3][3][Lmax/2]
  float* core = nullptr;    // [3 q][rho3][rho2][rho1]
};

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum (blockDim a multiple of 32, <= 1024); every thread gets the result
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;
}

}  // namespace

// QR of the generator matrix of (type, axis) = (j / 3, j % 3) by classical
// Gram-Schmidt with two re-orthogonalisation passes, FP64, one block per
// matrix.  Q column k at Q + (j M + k) glen (zero past m_p); R [j][M][M] upper
// triangular.  The generators of neighbouring nodes are numerically
// dependent (for large tau they all approach a multiple of the unit vector
// at d = 0): a column whose residual is below 1e-12 of its own norm is taken
// as in the span of the previous ones (R_kk = 0, zero Q column), so the
// residual noise is never normalised into a non-orthogonal direction; the
// factorisation then holds to 1e-12 of each column.
__global__ void __launch_bounds__(256) cmp_qr_kernel(int M, int glen, int m0, int m1, int m2, const double* gen,
                                                     double* Q, double* Rm) {
  __shared__ double coef[kMaxCompressTerms];
  __shared__ double red[32];
  const int j = blockIdx.x, axis = j % 3, type = j / 3;
  const int m = axis == 0 ? m0 : (axis == 1 ? m1 : m2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* Qj = Q + (size_t)j * M * glen;
  double* R = Rm + (size_t)j * M * M;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) R[i] = 0.0;
  for (int k = 0; k < M; ++k) {
    double* v = Qj + (size_t)k * glen;
    const double* a = gen + (((size_t)k * 2 + type) * 3 + axis) * glen;
    double a2 = 0.0;
    for (int e = threadIdx.x; e < glen; e += blockDim.x) {
      const double x = e < m ? a[e] : 0.0;
      v[e] = x;
      a2 += x * x;
    }
    const double anrm = sqrt(block_sum(a2, red));
    for (int pass = 0; pass < 3; ++pass) {
      for (int b = warp; b < k; b += nw) {
        const double* qb = Qj + (size_t)b * glen;
        double acc = 0.0;
        for (int e = lane; e < m; e += 32) acc += qb[e] * v[e];
        acc = warp_sum(acc);
        if (lane == 0) coef[b] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        double t = v[e];
        for (int b = 0; b < k; ++b) t -= coef[b] * Qj[(size_t)b * glen + e];
        v[e] = t;
      }
      if (threadIdx.x < k) R[threadIdx.x * M + k] += coef[threadIdx.x];
      __syncthreads();
    }
    double s2 = 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) s2 += v[e] * v[e];
    double nrm = sqrt(block_sum(s2, red));
    if (nrm <= 1e-12 * anrm) nrm = 0.0;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) v[e] *= inv;
    if (threadIdx.x == 0) R[k * M + k] = nrm;
    __syncthreads();
  }
}

// Symmetric eigen-decomposition of A (n x n, n even, leading dimension n, in
// shared memory) by cyclic Jacobi with a round-robin ordering (n/2 disjoint
// rotations per round): on return A is diagonal (the eigenvalues) and V holds
// the eigenvectors in its columns.  Each rotation G = [[c, s], [-s, c]] in
// rows/columns (p, q) zeroes a_pq with t = sgn(theta) / (|theta| + sqrt(1 + theta^2)),
// theta = (a_qq - a_pp) / (2 a_pq).  Stops when the off-diagonal part is below
// 1e-15 of the norm (squared: 1e-30) or after 30 sweeps.
__device__ void jacobi_eigen(double* A, double* V, int n, double* red) {
  __shared__ double rc[32], rs[32];
  __shared__ int rp[32], rq[32];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const double x = A[i] * A[i];
      all += x;
      if (i / n != i % n) off += x;
    }
    off = block_sum(off, red);
    all = block_sum(all, red);
    if (!(off > 1e-30 * all)) break;
    for (int round = 0; round < n - 1; ++round) {
      if (threadIdx.x < n / 2) {
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + round) % (n - 1); };
        int p = pos(threadIdx.x), q = pos(n - 1 - threadIdx.x);
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const double apq = A[p * n + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
          const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        rp[threadIdx.x] = p;
        rq[threadIdx.x] = q;
        rc[threadIdx.x] = c;
        rs[threadIdx.x] = s;
      }
      __syncthreads();
      const int half = n / 2;
      for (int idx = threadIdx.x; idx < half * n; idx += blockDim.x) {  // rows p, q
        const int r = idx / n, col = idx % n;
        const int p = rp[r], q = rq[r];
        const double c = rc[r], s = rs[r];
        const double ap = A[p * n + col], aq = A[q * n + col];
        A[p * n + col] = c * ap - s * aq;
        A[q * n + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < half * n; idx += blockDim.x) {  // columns p, q of A and V
        const int r = idx / n, row = idx % n;
        const int p = rp[r], q = rq[r];
        const double c = rc[r], s = rs[r];
        const double ap = A[row * n + p], aq = A[row * n + q];
        A[row * n + p] = c * ap - s * aq;
        A[row * n + q] = s * ap + c * aq;
        const double vp = V[row * n + p], vq = V[row * n + q];
        V[row * n + p] = c * vp - s * vq;
        V[row * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// S_p into A (n x n, zero past M):  S = R_p Lam (H_s o H_r) Lam R_p^T with
// H_x = B_x^T B_x, B_x = V_x^T R_x (V_x [M][M] column-major in its first rho_x
// columns) or B_x = R_x when V_x is NULL.  R matrices [M][M] row-major, upper
// triangular.  X and T are scratch (n x n).
__device__ void mode_matrix(int M, int n, const double* Rp, const double* Rs, const double* Rr, const double* Vs,
                            int rho_s, const double* Vr, int rho_r, const double* lam, double* X, double* T,
                            double* A) {
  for (int pass = 0; pass < 2; ++pass) {
    const double* R = pass ? Rr : Rs;
    const double* V = pass ? Vr : Vs;
    const int rho = V ? (pass ? rho_r : rho_s) : M;
    for (int idx = threadIdx.x; idx < rho * M; idx += blockDim.x) {  // B_x into T
      const int i = idx / M, a = idx % M;
      double b = 0.0;
      if (V) {
        for (int k = 0; k < M; ++k) b += V[k * M + i] * R[k * M + a];
      } else {
        b = R[i * M + a];
      }
      T[i * n + a] = b;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int a = idx / n, b = idx % n;
      double h = 0.0;
      if (a < M && b < M)
        for (int i = 0; i < rho; ++i) h += T[i * n + a] * T[i * n + b];
      X[idx] = pass ? X[idx] * h * lam[a < M ? a : 0] * lam[b < M ? b : 0] : h;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {  // T = R_p X
    const int i = idx / n, b = idx % n;
    double t = 0.0;
    if (i < M && b < M)
      for (int a = i; a < M; ++a) t += Rp[i * M + a] * X[a * n + b];
    T[idx] = t;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {  // A = T R_p^T
    const int i = idx / n, j = idx % n;
    double t = 0.0;
    if (i < M && j < M)
      for (int b = j; b < M; ++b) t += T[i * n + b] * Rp[j * M + b];
    A[idx] = t;
  }
  __syncthreads();
}

// Eigenvalues of A (after jacobi_eigen) in descending order of the first M
// indices (a padding index stays decoupled), eigenvectors written column i of
// Vout [M][M].  Returns nothing; eig gets M values.
__device__ void sorted_out(int M, int n, const double* A, const double* V, double* eig, double* Vout) {
  __shared__ int ord[kMaxCompressTerms];
  if (threadIdx.x == 0) {
    for (int i = 0; i < M; ++i) ord[i] = i;
    for (int i = 0; i < M; ++i) {
      int best = i;
      for (int j = i + 1; j < M; ++j)
        if (A[ord[j] * n + ord[j]] > A[ord[best] * n + ord[best]]) best = j;
      const int t = ord[i];
      ord[i] = ord[best];
      ord[best] = t;
    }
  }
  __syncthreads();
  if (eig)
    for (int i = threadIdx.x; i < M; i += blockDim.x) eig[i] = A[ord[i] * n + ord[i]];
  for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
    const int k = idx / M, i = idx % M;
    Vout[idx] = V[k * n + ord[i]];
  }
  __syncthreads();
}

__device__ __forceinline__ const double* r_of(const double* Rm, int M, int axis, int q) {
  return Rm + (size_t)((axis == q ? 1 : 0) * 3 + axis) * M * M;
}

// HOSVD of K^(q) (block q): eigen-decomposition of S_p with B_x = R_x, for p = 1..3.
__global__ void __launch_bounds__(256) cmp_hosvd_kernel(int M, int n, const double* Rm, const double* lam,
                                                        double* eig, double* Vfull) {
  extern __shared__ double smc[];
  __shared__ double red[32];
  double *X = smc, *T = X + n * n, *A = T + n * n, *V = A + n * n;
  const int q = blockIdx.x;
  for (int p = 0; p < 3; ++p) {
    const int s = (p + 1) % 3, r = (p + 2) % 3;
    mode_matrix(M, n, r_of(Rm, M, p, q), r_of(Rm, M, s, q), r_of(Rm, M, r, q), nullptr, 0, nullptr, 0, lam, X, T, A);
    jacobi_eigen(A, V, n, red);
    sorted_out(M, n, A, V, eig + (size_t)(q * 3 + p) * M, Vfull + (size_t)(q * 3 + p) * M * M);
  }
}

// HOOI sweeps of Alg. 1 at ranks rho (block q) from the HOSVD start in Vcur,
// then the core C[i3][i2][i1] = sum_k lam_k b_{1k}[i1] b_{2k}[i2] b_{3k}[i3].
__global__ void __launch_bounds__(256) cmp_hooi_kernel(int M, int n, int rho0, int rho1, int rho2, int sweeps,
                                                       const double* Rm, const double* lam, double* Vcur,
                                                       float* core) {
  extern __shared__ double smc[];
  __shared__ double red[32];
  double *X = smc, *T = X + n * n, *A = T + n * n, *V = A + n * n;
  const int q = blockIdx.x;
  const int rho[3] = {rho0, rho1, rho2};
  double* Vq = Vcur + (size_t)q * 3 * M * M;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int p = 0; p < 3; ++p) {
      const int s = (p + 1) % 3, r = (p + 2) % 3;
      mode_matrix(M, n, r_of(Rm, M, p, q), r_of(Rm, M, s, q), r_of(Rm, M, r, q), Vq + (size_t)s * M * M, rho[s],
                  Vq + (size_t)r * M * M, rho[r], lam, X, T, A);
      jacobi_eigen(A, V, n, red);
      sorted_out(M, n, A, V, nullptr, Vq + (size_t)p * M * M);
    }
  }
  // b_p = V_p^T R_p into X (p = 0), T (1), A (2): [rho_p][M] at leading dimension n
  double* B[3] = {X, T, A};
  for (int p = 0; p < 3; ++p) {
    const double* R = r_of(Rm, M, p, q);
    const double* Vp = Vq + (size_t)p * M * M;
    for (int idx = threadIdx.x; idx < rho[p] * M; idx += blockDim.x) {
      const int i = idx / M, a = idx % M;
      double b = 0.0;
      for (int k = 0; k < M; ++k) b += Vp[k * M + i] * R[k * M + a];
      B[p][i * n + a] = b;
    }
  }
  __syncthreads();
  const int total = rho0 * rho1 * rho2;
  float* Cq = core + (size_t)q * total;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int i1 = idx % rho0, i2 = (idx / rho0) % rho1, i3 = idx / (rho0 * rho1);
    double c = 0.0;
    for (int k = 0; k < M; ++k) c += lam[k] * X[i1 * n + k] * T[i2 * n + k] * A[i3 * n + k];
    Cq[idx] = (float)c;
  }
}

// Compressed generators U_p^(q) = Q_{type,p} V_p^(q): row (i, q, p) of cgen, i < rho_p, e < m_p.
__global__ void cmp_gen_kernel(int M, int glen, int rho0, int rho1, int rho2, int m0, int m1, int m2,
                               const double* Q, const double* Vcur, double* cgen) {
  const int rho[3] = {rho0, rho1, rho2};
  const int mm[3] = {m0, m1, m2};
  const int rmax = max(rho0, max(rho1, rho2));
  const long total = (long)rmax * 9 * glen;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int e = (int)(idx % glen);
    const long row = idx / glen;  // (i * 3 + q) * 3 + p
    const int p = (int)(row % 3), q = (int)((row / 3) % 3), i = (int)(row / 9);
    double v = 0.0;
    if (i < rho[p] && e < mm[p]) {
      const int j = (p == q ? 1 : 0) * 3 + p;
      const double* Qj = Q + (size_t)j * M * glen;
      const double* Vp = Vcur + (size_t)(q * 3 + p) * M * M;
      for (int k = 0; k < M; ++k) v += Qj[(size_t)k * glen + e] * Vp[k * M + i];
    }
    cgen[idx] = v;
  }
}

// out_core[b][q][(i3 r3 + l3)][(i2 r2 + l2)][(i1 r1 + l1)] = C^(q)[i3][i2][i1] G[b][q][l3][l2][l1]
__global__ void cmp_core_kernel(int batch, int rho0, int rho1, int rho2, int r0, int r1, int r2, const float* C,
                                const float* G, float* out) {
  const long per = (long)rho0 * r0 * rho1 * r1 * rho2 * r2;
  const long total = (long)batch * 3 * per;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    long t = idx % per;
    const long bq = idx / per;
    const int q = (int)(bq % 3);
    const int c1 = (int)(t % ((long)rho0 * r0));
    t /= (long)rho0 * r0;
    const int c2 = (int)(t % ((long)rho1 * r1));
    const int c3 = (int)(t / ((long)rho1 * r1));
    const int i1 = c1 / r0, l1 = c1 % r0, i2 = c2 / r1, l2 = c2 % r1, i3 = c3 / r2, l3 = c3 % r2;
    const float cv = C[(size_t)q * rho0 * rho1 * rho2 + ((size_t)i3 * rho1 + i2) * rho0 + i1];
    const float gv = G[(size_t)bq * r0 * r1 * r2 + ((size_t)l3 * r1 + l2) * r0 + l1];
    out[idx] = cv * gv;
  }
}

// ---------------------------------------------------------------- recompression of phi
//
// Alg. 2's last step ("approximate summation with tolerance tol") for the
// output of demag_apply_tucker_compressed: phi = sum_q [[E_q; W_q1, W_q2, W_q3]]
// with E_q = C^(q) (x) G^(q) (ranks R_p = rho_p r_p per component) is brought to
// one Tucker tensor [[C; U_1, U_2, U_3]].  Range of each unfolding: phi_(p)
// applied to k Khatri-Rao test vectors (+-1 entries from a counter hash), QR
// (the CGS kernel above); core C = phi x_p U_p^T; the projection error is
// ||phi||^2 - ||C||^2 exactly (U_p orthonormal), with
// ||phi||^2 = sum_{q,q'} <E_q, E_q' x_p (W_qp^T W_q'p)>; then an HOSVD of the
// small core truncated so that the total error stays below tol ||phi||.
// FP64 throughout.

// Column-major [cols][m] matrix from the compressed factors of one item:
// W_qp column (i r_p + l) = row (i, q, l) of mode block p.
__global__ void rc_gather_kernel(int q, int p, int rho, int r, int n, const float* block, double* W) {
  const long total = (long)rho * r * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int e = (int)(idx % n);
    const long c = idx / n;
    const int i = (int)(c / r), l = (int)(c % r);
    W[idx] = (double)block[(((size_t)i * 3 + q) * r + l) * n + e];
  }
}

// E[(i3 r3 + l3)][(i2 r2 + l2)][(i1 r1 + l1)] = C[i3][i2][i1] G[l3][l2][l1] (one component)
__global__ void rc_core_kernel(int rho0, int rho1, int rho2, int r0, int r1, int r2, const float* C, const float* G,
                               double* E) {
  const long R0 = (long)rho0 * r0, R1 = (long)rho1 * r1, total = R0 * R1 * rho2 * r2;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const long c1 = idx % R0, c2 = (idx / R0) % R1, c3 = idx / (R0 * R1);
    const int i1 = (int)(c1 / r0), l1 = (int)(c1 % r0), i2 = (int)(c2 / r1), l2 = (int)(c2 % r1);
    const int i3 = (int)(c3 / r2), l3 = (int)(c3 % r2);
    E[idx] = (double)C[((size_t)i3 * rho1 + i2) * rho0 + i1] * (double)G[((size_t)l3 * r1 + l2) * r0 + l1];
  }
}

// out = X x_p Mx (Eq. modemul): X [d2][d1][d0] (d0 fastest), Mx [e][d_p] row-major; out has d_p -> e.
// With acc the result is added to out.
__global__ void rc_mode_kernel(int d0, int d1, int d2, int p, int e, const double* X, const double* Mx, double* out,
                               int acc) {
  const int o0 = p == 0 ? e : d0, o1 = p == 1 ? e : d1, o2 = p == 2 ? e : d2;
  const long total = (long)o0 * o1 * o2;
  const int dp = p == 0 ? d0 : (p == 1 ? d1 : d2);
  const long stride = p == 0 ? 1 : (p == 1 ? d0 : (long)d0 * d1);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int a0 = (int)(idx % o0), a1 = (int)((idx / o0) % o1), a2 = (int)(idx / ((long)o0 * o1));
    const int a = p == 0 ? a0 : (p == 1 ? a1 : a2);
    const long base = (p == 0 ? 0 : a0) + (long)(p == 1 ? 0 : a1) * d0 + (long)(p == 2 ? 0 : a2) * d0 * d1;
    double t = 0.0;
    for (int b = 0; b < dp; ++b) t += Mx[(long)a * dp + b] * X[base + b * stride];
    out[idx] = acc ? out[idx] + t : t;
  }
}

// G[i][j] = sum_e A[i m + e] B[j m + e] (column-major A [a][m], B [b][m]); one warp per entry
__global__ void rc_gram_kernel(int m, int a, int b, const double* A, const double* B, double* G) {
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long w = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); w < (long)a * b; w += warps) {
    const int i = (int)(w / b), j = (int)(w % b);
    double t = 0.0;
    for (int e = lane; e < m; e += 32) t += A[(long)i * m + e] * B[(long)j * m + e];
    t = warp_sum(t);
    if (lane == 0) G[w] = t;
  }
}

// +-1 test entry of (mode, row e, sample j) from a counter hash (splitmix-style mixing)
__device__ __forceinline__ double rc_sign(unsigned long long seed, int mode, int e, int j) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (((unsigned long long)mode << 48) ^
                                                         ((unsigned long long)j << 32) ^ (unsigned)e);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (z & 1ull) ? 1.0 : -1.0;
}

// A[c][j] = sum_e W[c m + e] omega_mode(e, j): the test vectors seen through a factor
__global__ void rc_probe_kernel(int m, int cols, int k, int mode, unsigned long long seed, const double* W, double* A) {
  const long total = (long)cols * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / k), j = (int)(idx % k);
    double t = 0.0;
    for (int e = 0; e < m; ++e) t += W[(long)c * m + e] * rc_sign(seed, mode, e, j);
    A[idx] = t;
  }
}

// Z[i][j] = sum_{a, b} E[.. i ..] As[a][j] Ar[b][j], the core contracted on modes s, r
// with sample j of the test vectors (Khatri-Rao test); E dims R0, R1, R2 (R0 fastest)
__global__ void rc_sketch_kernel(int R0, int R1, int R2, int p, int k, const double* E, const double* As,
                                 const double* Ar, double* Z) {
  const int Rd[3] = {R0, R1, R2};
  const int s = (p + 1) % 3, r = (p + 2) % 3;
  const long st[3] = {1, R0, (long)R0 * R1};
  const long total = (long)Rd[p] * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / k), j = (int)(idx % k);
    double t = 0.0;
    for (int b = 0; b < Rd[r]; ++b) {
      double u = 0.0;
      const double* row = E + i * st[p] + b * st[r];
      for (int a = 0; a < Rd[s]; ++a) u += row[a * st[s]] * As[(long)a * k + j];
      t += u * Ar[(long)b * k + j];
    }
    Z[idx] = t;
  }
}

// Y[j][e] (column-major [k][n]) += sum_c W[c n + e] Z[c][j]
__global__ void rc_range_kernel(int n, int cols, int k, const double* W, const double* Z, double* Y, int acc) {
  const long total = (long)k * n;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / n), e = (int)(idx % n);
    double t = 0.0;
    for (int c = 0; c < cols; ++c) t += W[(long)c * n + e] * Z[(long)c * k + j];
    Y[idx] = acc ? Y[idx] + t : t;
  }
}

// QR of a column-major [M][m] matrix by the same CGS (three passes, 1e-12 drop) as cmp_qr_kernel
__global__ void __launch_bounds__(256) rc_qr_kernel(int M, int m, const double* A, double* Q, double* R) {
  __shared__ double coef[kMaxCompressTerms];
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) R[i] = 0.0;
  for (int k = 0; k < M; ++k) {
    double* v = Q + (size_t)k * m;
    double a2 = 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      const double x = A[(size_t)k * m + e];
      v[e] = x;
      a2 += x * x;
    }
    const double anrm = sqrt(block_sum(a2, red));
    for (int pass = 0; pass < 3; ++pass) {
      for (int b = warp; b < k; b += nw) {
        const double* qb = Q + (size_t)b * m;
        double acc = 0.0;
        for (int e = lane; e < m; e += 32) acc += qb[e] * v[e];
        acc = warp_sum(acc);
        if (lane == 0) coef[b] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < m; e += blockDim.x) {
        double t = v[e];
        for (int b = 0; b < k; ++b) t -= coef[b] * Q[(size_t)b * m + e];
        v[e] = t;
      }
      if (threadIdx.x < k) R[threadIdx.x * M + k] += coef[threadIdx.x];
      __syncthreads();
    }
    double s2 = 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) s2 += v[e] * v[e];
    double nrm = sqrt(block_sum(s2, red));
    if (nrm <= 1e-12 * anrm) nrm = 0.0;
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int e = threadIdx.x; e < m; e += blockDim.x) v[e] *= inv;
    if (threadIdx.x == 0) R[k * M + k] = nrm;
    __syncthreads();
  }
}

// sum of x[i] y[i] into *out (FP64, one atomic per block)
__global__ void rc_dot_kernel(long count, const double* x, const double* y, double* out) {
  __shared__ double red[32];
  double t = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    t += x[i] * y[i];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(out, s);
  }
}

// HOSVD of the small core (dims k0, k1, k2 <= 64, k0 fastest; one block): for
// each mode the unfolding Gram (k_p x k_p, padded to n even), Jacobi,
// eigenvalues (descending) into eig + 64 p and eigenvectors into V + 4096 p
// ([k_p][k_p], column i = vector i).
__global__ void __launch_bounds__(256) rc_core_hosvd_kernel(int k0, int k1, int k2, int n, const double* C,
                                                            double* eig, double* V) {
  extern __shared__ double smc[];
  __shared__ double red[32];
  double *A = smc, *Vs = A + n * n;
  const int kd[3] = {k0, k1, k2};
  const long st[3] = {1, k0, (long)k0 * k1};
  for (int p = 0; p < 3; ++p) {
    const int s = (p + 1) % 3, r = (p + 2) % 3, kp = kd[p];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int a = idx / n, b = idx % n;
      double t = 0.0;
      if (a < kp && b < kp)
        for (int x = 0; x < kd[s]; ++x)
          for (int y = 0; y < kd[r]; ++y) {
            const long off = x * st[s] + y * st[r];
            t += C[off + a * st[p]] * C[off + b * st[p]];
          }
      A[idx] = t;
    }
    __syncthreads();
    jacobi_eigen(A, Vs, n, red);
    sorted_out(kp, n, A, Vs, eig + 64 * p, V + 4096 * p);
  }
}

// ---------------------------------------------------------------- TT rounding of phi
//
// App. C: the potential of a TT magnetization is a sum of T = 3M trains
// (w_t G1_t G2_t G3_t, ranks r1, r2 each).  Rounding to tolerance tol: the
// range of the first unfolding is sampled with Khatri-Rao products of +-1
// test vectors (through the train: Y1 = sum_t w_t G1_t (G2_t x omega2) (G3_t omega3)),
// QR'd (Q1); the projected train's (1,2)-unfolding is sampled with omega3 and
// QR'd (Q2); the last core is Z = Q2^T (Q1^T phi).  The projection error
// ||phi||^2 - ||Z||^2 is exact (||phi||^2 from the pairwise Grams of the terms);
// samples grow (16, 32, 64) until it is below tol/2.  Then the small train
// [Q1, Q2, Z] is truncated as in TT-SVD: the mode-1 Gram (Jacobi), a QR of the
// truncated middle core, the Gram of the new last core; each truncation keeps
// its discarded part within half of the remaining budget.  FP64 throughout.

__global__ void rc_f2d_kernel(long count, const float* x, double* y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// ||phi||^2 = sum_{t,t'} w_t w_t' sum GA[(t a1),(t' b1)] GB[(t a1 a2),(t' b1 b2)] GC[(t a2),(t' b2)]
__global__ void tt_norm_kernel(int T, int ra, int rb, const double* w, const double* GA, const double* GB,
                               const double* GC, double* out) {
  __shared__ double red[32];
  const long na = (long)T * ra, nb = (long)T * ra * rb, nc = (long)T * rb;
  double acc = 0.0;
  for (long pr = blockIdx.x * (long)blockDim.x + threadIdx.x; pr < (long)T * T; pr += (long)gridDim.x * blockDim.x) {
    const int t = (int)(pr / T), u = (int)(pr % T);
    double s = 0.0;
    for (int a1 = 0; a1 < ra; ++a1)
      for (int b1 = 0; b1 < ra; ++b1) {
        const double ga = GA[((long)t * ra + a1) * na + (long)u * ra + b1];
        for (int a2 = 0; a2 < rb; ++a2)
          for (int b2 = 0; b2 < rb; ++b2)
            s += ga * GB[(((long)t * ra + a1) * rb + a2) * nb + ((long)u * ra + b1) * rb + b2] *
                 GC[((long)t * rb + a2) * nc + (long)u * rb + b2];
      }
    acc += w[t] * w[u] * s;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    atomicAdd(out, v);
  }
}

// h[(t a1)][j] = w_t sum_a2 BW[(t a1 a2)][j] CW[(t a2)][j]
__global__ void tt_h_kernel(int T, int ra, int rb, int k, const double* w, const double* BW, const double* CW,
                            double* h) {
  const long total = (long)T * ra * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % k);
    const long ta = idx / k;
    const int t = (int)(ta / ra);
    double s = 0.0;
    for (int a2 = 0; a2 < rb; ++a2) s += BW[(ta * rb + a2) * k + j] * CW[((long)t * rb + a2) * k + j];
    h[idx] = w[t] * s;
  }
}

// F[(t a1)][i2][j] = w_t sum_a2 B[(t a1 a2)][i2] CW[(t a2)][j]
__global__ void tt_f_kernel(int T, int ra, int rb, int n2, int k, const double* w, const double* B, const double* CW,
                            double* F) {
  const long total = (long)T * ra * n2 * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % k);
    const long r = idx / k;
    const int i2 = (int)(r % n2);
    const long ta = r / n2;
    const int t = (int)(ta / ra);
    double s = 0.0;
    for (int a2 = 0; a2 < rb; ++a2) s += B[(ta * rb + a2) * n2 + i2] * CW[((long)t * rb + a2) * k + j];
    F[idx] = w[t] * s;
  }
}

// Y2[j][(a i2)] = sum_c AP[a][c] F[c][i2][j], c = (t a1) < cols; Y2 column-major [k][k1 n2]
__global__ void tt_y2_kernel(int k1, int n2, int k, int cols, const double* AP, const double* F, double* Y2) {
  const long m = (long)k1 * n2, total = m * k;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / m);
    const long row = idx % m;
    const int a = (int)(row / n2), i2 = (int)(row % n2);
    double s = 0.0;
    for (int c = 0; c < cols; ++c) s += AP[(long)a * cols + c] * F[((long)c * n2 + i2) * k + j];
    Y2[idx] = s;
  }
}

// Pm[c][i2][j] = sum_a Q2[j][(a i2)] AP[a][c]
__global__ void tt_p_kernel(int k1, int n2, int k2, int cols, const double* Q2, const double* AP, double* Pm) {
  const long total = (long)cols * n2 * k2;
  const long m = (long)k1 * n2;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % k2);
    const long r = idx / k2;
    const int i2 = (int)(r % n2);
    const long c = r / n2;
    double s = 0.0;
    for (int a = 0; a < k1; ++a) s += Q2[(long)j * m + (long)a * n2 + i2] * AP[(long)a * cols + c];
    Pm[idx] = s;
  }
}

// wE[(t a2)][j] = w_t sum_{a1, i2} Pm[(t a1)][i2][j] B[(t a1 a2)][i2]
__global__ void tt_e_kernel(int T, int ra, int rb, int n2, int k2, const double* w, const double* Pm, const double* B,
                            double* wE) {
  const long total = (long)T * rb * k2;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % k2);
    const long tb = idx / k2;
    const int t = (int)(tb / rb), a2 = (int)(tb % rb);
    double s = 0.0;
    for (int a1 = 0; a1 < ra; ++a1) {
      const long c = (long)t * ra + a1;
      const double* brow = B + (c * rb + a2) * n2;
      for (int i2 = 0; i2 < n2; ++i2) s += Pm[(c * n2 + i2) * k2 + j] * brow[i2];
    }
    wE[idx] = w[t] * s;
  }
}

// out[(b i2)][j] = sum_a Wm[a][b] V[j][(a i2)]  -> stored column-major [k2][rb1 n2] (V' = W1^T x_1 V)
__global__ void tt_vprime_kernel(int k1, int rb1, int n2, int k2, const double* Wm, const double* V, double* out) {
  const long m = (long)rb1 * n2, total = m * k2;
  const long mv = (long)k1 * n2;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
    const int j = (int)(idx / m);
    const long row = idx % m;
    const int b = (int)(row / n2), i2 = (int)(row % n2);
    double s = 0.0;
    for (int a = 0; a < k1; ++a) s += Wm[(long)a * rb1 + b] * V[(long)j * mv + (long)a * n2 + i2];
    out[idx] = s;
  }
}

// M1[a][b] = sum_{j, i2} V[j][(a i2)] VZ[j][(b i2)] with VZ = V ZZ (the mode-1 Gram of [V; Z])
__global__ void tt_m1_kernel(int k1, int n2, int k2, const double* V, const double* VZ, double* M1) {
  const long m = (long)k1 * n2;
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  for (long wI = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); wI < (long)k1 * k1; wI += warps) {
    const int a = (int)(wI / k1), b = (int)(wI % k1);
    double s = 0.0;
    for (long x = lane; x < (long)k2 * n2; x += 32) {
      const int j = (int)(x / n2), i2 = (int)(x % n2);
      s += V[(long)j * m + (long)a * n2 + i2] * VZ[(long)j * m + (long)b * n2 + i2];
    }
    s = warp_sum(s);
    if (lane == 0) M1[wI] = s;
  }
}

// eigen-decomposition of one k x k symmetric matrix (one block, k <= 64): eig desc, V [k][k]
__global__ void __launch_bounds__(256) rc_eig_kernel(int k, int n, const double* S, double* eig, double* V) {
  extern __shared__ double smc[];
  __shared__ double red[32];
  double *A = smc, *Vs = A + n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int a = idx / n, b = idx % n;
    A[idx] = (a < k && b < k) ? S[(long)a * k + b] : 0.0;
  }
  __syncthreads();
  jacobi_eigen(A, Vs, n, red);
  sorted_out(k, n, A, Vs, eig, V);
}

void compress_destroy(demag_plan* P) {
  Compressed* C = static_cast<Compressed*>(P->cmp);
  if (!C) return;
  cudaFree(C->cgen);
  cudaFree(C->csym);
  cudaFree(C->cpair);
  cudaFree(C->core);
  delete C;
  P->cmp = nullptr;
}

bool compressed_view(const demag_plan* P, CompressedView* v) {
  const Compressed* C = static_cast<const Compressed*>(P ? P->cmp : nullptr);
  if (!C) return false;
  for (int p = 0; p < 3; ++p) v->rho[p] = C->rho[p];
  v->cpair = C->cpair;
  v->core = C->core;
  return true;
}

demag_status launch_core_kron(demag_plan* P, int batch, const int r[3], const float* G, float* out, cudaStream_t st) {
  const Compressed* C = static_cast<const Compressed*>(P->cmp);
  const long total = (long)batch * 3 * C->rho[0] * r[0] * C->rho[1] * r[1] * C->rho[2] * r[2];
  long blocks = (total + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  DEMAG_LAUNCH(P, kFamMisc, st,
               cmp_core_kernel<<<(int)blocks, 256, 0, st>>>(batch, C->rho[0], C->rho[1], C->rho[2], r[0], r[1], r[2],
                                                            C->core, G, out));
  DEMAG_LAUNCHED(P, "cmp_core_kernel");
  return DEMAG_OK;
}

}  // namespace demag

using namespace demag;

// tail[r] = sum_{i >= r} sigma_i^2 of descending eigenvalues sigma^2; the
// smallest r with tail[r] <= (tol^2 / 3) sum sigma^2 (at least 1).
static int truncation_rank(const double* sig2, int M, double tol) {
  double total = 0.0;
  for (int i = 0; i < M; ++i) total += sig2[i] > 0.0 ? sig2[i] : 0.0;
  const double bound = tol * tol / 3.0 * total;
  double tail = total;
  for (int r = 1; r <= M; ++r) {
    tail -= sig2[r - 1] > 0.0 ? sig2[r - 1] : 0.0;
    if (tail <= bound) return r;
  }
  return M;
}

extern "C" demag_status demag_compress_kernel(demag_plan* P, double tol, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_compress_kernel: plan is NULL");
  demag_status u = require_uniform(P, "demag_compress_kernel");
  if (u != DEMAG_OK) return u;
  if (!(tol > 0.0 && tol < 1.0)) return set_error(P, DEMAG_EINVAL, "demag_compress_kernel: tol must be in (0, 1)");
  if (!P->sympair || !P->twid[0])
    return set_error(P, DEMAG_EUNSUPPORTED, "demag_compress_kernel: n_p up to %d supported by the FFT path",
                     1 << kMaxFFTLog);
  if (P->M > kMaxCompressTerms)
    return set_error(P, DEMAG_EUNSUPPORTED, "demag_compress_kernel: M = %d terms, at most %d (R <= %d) supported",
                     P->M, kMaxCompressTerms, 2 * kMaxCompressTerms + 1);
  cudaStream_t st = (cudaStream_t)stream;
  const int M = P->M, glen = P->glen, n = M + (M & 1);
  const int m[3] = {2 * P->n[0] - 1, 2 * P->n[1] - 1, 2 * P->n[2] - 1};
  double *Q = nullptr, *R = nullptr, *eig = nullptr, *Vfull = nullptr, *Vcur = nullptr;
  Compressed* C = new (std::nothrow) Compressed();
  if (!C) return set_error(P, DEMAG_ENOMEM, "host allocation failed");
  auto cleanup = [&]() {
    cudaFree(Q);
    cudaFree(R);
    cudaFree(eig);
    cudaFree(Vfull);
    cudaFree(Vcur);
  };
  auto fail = [&](demag_status s) {
    cleanup();
    cudaFree(C->cgen);
    cudaFree(C->csym);
    cudaFree(C->cpair);
    cudaFree(C->core);
    delete C;
    return s;
  };
#define CMP_CUDA(call)                                          \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return fail(cuda_error(P, e_, #call)); \
  } while (0)
  CMP_CUDA(cudaMalloc(&Q, sizeof(double) * 6 * M * glen));
  CMP_CUDA(cudaMalloc(&R, sizeof(double) * 6 * M * M));
  CMP_CUDA(cudaMalloc(&eig, sizeof(double) * 9 * M));
  CMP_CUDA(cudaMalloc(&Vfull, sizeof(double) * 9 * M * M));
  CMP_CUDA(cudaMalloc(&Vcur, sizeof(double) * 9 * M * M));
  const size_t smem = sizeof(double) * 4 * n * n;
  static unsigned long long attr = 0;  // devices whose kernel attributes are set
  int dev = 0;
  CMP_CUDA(cudaGetDevice(&dev));
  if (!(attr & (1ull << (dev & 63)))) {
    CMP_CUDA(cudaFuncSetAttribute(cmp_hosvd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 64 * 64 * 8));
    CMP_CUDA(cudaFuncSetAttribute(cmp_hooi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * 64 * 64 * 8));
    attr |= 1ull << (dev & 63);
  }
  DEMAG_LAUNCH(P, kFamSetup, st, cmp_qr_kernel<<<6, 256, 0, st>>>(M, glen, m[0], m[1], m[2], P->gen64, Q, R));
  CMP_CUDA(cudaGetLastError());
  DEMAG_LAUNCH(P, kFamSetup, st, cmp_hosvd_kernel<<<3, 256, smem, st>>>(M, n, R, P->scale, eig, Vfull));
  CMP_CUDA(cudaGetLastError());
  std::vector<double> eh((size_t)9 * M);
  CMP_CUDA(cudaMemcpyAsync(eh.data(), eig, sizeof(double) * 9 * M, cudaMemcpyDeviceToHost, st));
  CMP_CUDA(cudaStreamSynchronize(st));
  for (int p = 0; p < 3; ++p) {
    C->rho[p] = 1;
    for (int q = 0; q < 3; ++q) C->rho[p] = std::max(C->rho[p], truncation_rank(&eh[(size_t)(q * 3 + p) * M], M, tol));
  }
  C->tol = tol;
  CMP_CUDA(cudaMemcpyAsync(Vcur, Vfull, sizeof(double) * 9 * M * M, cudaMemcpyDeviceToDevice, st));
  CMP_CUDA(cudaMalloc(&C->core, sizeof(float) * 3 * C->rho[0] * C->rho[1] * C->rho[2]));
  DEMAG_LAUNCH(P, kFamSetup, st,
               cmp_hooi_kernel<<<3, 256, smem, st>>>(M, n, C->rho[0], C->rho[1], C->rho[2], 4, R, P->scale, Vcur,
                                                     C->core));
  CMP_CUDA(cudaGetLastError());
  const int rmax = std::max(C->rho[0], std::max(C->rho[1], C->rho[2]));
  CMP_CUDA(cudaMalloc(&C->cgen, sizeof(double) * (size_t)rmax * 9 * glen));
  {
    const long total = (long)rmax * 9 * glen;
    long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 cmp_gen_kernel<<<(int)blocks, 256, 0, st>>>(M, glen, C->rho[0], C->rho[1], C->rho[2], m[0], m[1], m[2],
                                                             Q, Vcur, C->cgen));
    CMP_CUDA(cudaGetLastError());
  }
  const int symstride = P->Lmax / 2 + 1, pairstride = P->Lmax / 2;
  CMP_CUDA(cudaMalloc(&C->csym, sizeof(float) * (size_t)rmax * 9 * symstride));
  CMP_CUDA(cudaMemsetAsync(C->csym, 0, sizeof(float) * (size_t)rmax * 9 * symstride, st));
  CMP_CUDA(cudaMalloc(&C->cpair, sizeof(float2) * (size_t)rmax * 9 * pairstride));
  for (int p = 0; p < 3; ++p) {
    dispatch_symbol(P, p, C->rho[p], 3, C->cgen, C->csym, st);
    CMP_CUDA(cudaGetLastError());
    const int N = P->L[p] / 2;
    const long total = (long)C->rho[p] * 3 * N;
    long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 sympair_kernel<<<(int)blocks, 256, 0, st>>>(C->rho[p], 3, p, N, symstride, pairstride, C->csym,
                                                             C->cpair));
    CMP_CUDA(cudaGetLastError());
  }
  CMP_CUDA(cudaStreamSynchronize(st));
#undef CMP_CUDA
  cleanup();
  compress_destroy(P);
  P->cmp = C;
  return DEMAG_OK;
}

extern "C" demag_status demag_compressed_ranks(const demag_plan* plan, int rho[3]) {
  demag_plan* P = const_cast<demag_plan*>(plan);
  if (!P || !rho) return set_error(P, DEMAG_EINVAL, "demag_compressed_ranks: NULL argument");
  const Compressed* C = static_cast<const Compressed*>(P->cmp);
  if (!C) return set_error(P, DEMAG_EINVAL, "demag_compressed_ranks: no compressed kernel (demag_compress_kernel)");
  for (int p = 0; p < 3; ++p) rho[p] = C->rho[p];
  return DEMAG_OK;
}

extern "C" demag_status demag_copy_compressed(const demag_plan* plan, double* gen, float* core, void* stream) {
  demag_plan* P = const_cast<demag_plan*>(plan);
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_copy_compressed: plan is NULL");
  const Compressed* C = static_cast<const Compressed*>(P->cmp);
  if (!C) return set_error(P, DEMAG_EINVAL, "demag_copy_compressed: no compressed kernel (demag_compress_kernel)");
  cudaStream_t st = (cudaStream_t)stream;
  const int rmax = std::max(C->rho[0], std::max(C->rho[1], C->rho[2]));
  if (gen)
    DEMAG_CUDA(P, cudaMemcpyAsync(gen, C->cgen, sizeof(double) * (size_t)rmax * 9 * P->glen,
                                  cudaMemcpyDeviceToDevice, st));
  if (core)
    DEMAG_CUDA(P, cudaMemcpyAsync(core, C->core, sizeof(float) * 3 * C->rho[0] * C->rho[1] * C->rho[2],
                                  cudaMemcpyDeviceToDevice, st));
  DEMAG_CUDA(P, cudaStreamSynchronize(st));
  return DEMAG_OK;
}

static int rc_blocks(long total) {
  long b = (total + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (int)(b < 1 ? 1 : b);
}

extern "C" demag_status demag_recompress_tucker(demag_plan* P, const int r[3], const float* core, const float* V,
                                                double tol, int ranks_out[3], float* core_out, float* U_out,
                                                double* err_out, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_recompress_tucker: plan is NULL");
  if (!r || !core || !V || !ranks_out || !core_out || !U_out)
    return set_error(P, DEMAG_EINVAL, "demag_recompress_tucker: NULL pointer");
  if (!(tol > 0.0 && tol < 1.0)) return set_error(P, DEMAG_EINVAL, "demag_recompress_tucker: tol must be in (0, 1)");
  CompressedView cv;
  if (!compressed_view(P, &cv))
    return set_error(P, DEMAG_EINVAL, "demag_recompress_tucker: no compressed kernel (demag_compress_kernel)");
  for (int p = 0; p < 3; ++p)
    if (r[p] < 1) return set_error(P, DEMAG_EINVAL, "demag_recompress_tucker: r[%d] must be >= 1", p);
  cudaStream_t st = (cudaStream_t)stream;
  const int n[3] = {P->n[0], P->n[1], P->n[2]};
  int Rr[3];
  for (int p = 0; p < 3; ++p) Rr[p] = cv.rho[p] * r[p];
  const long Rtot = (long)Rr[0] * Rr[1] * Rr[2];
  long tmpn = Rtot;
  for (int p = 0; p < 3; ++p) tmpn = std::max(tmpn, (long)64 * Rr[(p + 1) % 3] * Rr[(p + 2) % 3]);
  tmpn = std::max(tmpn, (long)64 * 64 * 64);
  long wsize = 0;
  long woff[3][3];
  for (int q = 0; q < 3; ++q)
    for (int p = 0; p < 3; ++p) {
      woff[q][p] = wsize;
      wsize += (long)Rr[p] * n[p];
    }
  const int Rmax = std::max(Rr[0], std::max(Rr[1], Rr[2]));
  const int nmax = std::max(n[0], std::max(n[1], n[2]));
  std::vector<void*> owned;
  auto alloc = [&](double** ptr, long count) {
    cudaError_t e = cudaMalloc(ptr, sizeof(double) * (size_t)std::max(count, 1L));
    if (e == cudaSuccess) owned.push_back(*ptr);
    return e;
  };
  auto release = [&]() {
    for (void* q : owned) cudaFree(q);
    owned.clear();
  };
  double *W, *E, *T1, *T2, *G, *Y[3], *Q[3], *Rq, *A1, *A2, *Z, *B, *Ch, *acc, *eig, *Vh, *Mt;
  cudaError_t e = cudaSuccess;
  if ((e = alloc(&W, wsize)) != cudaSuccess || (e = alloc(&E, 3 * Rtot)) != cudaSuccess ||
      (e = alloc(&T1, tmpn)) != cudaSuccess || (e = alloc(&T2, tmpn)) != cudaSuccess ||
      (e = alloc(&G, (long)Rmax * Rmax)) != cudaSuccess || (e = alloc(&Rq, 64 * 64)) != cudaSuccess ||
      (e = alloc(&A1, (long)Rmax * 64)) != cudaSuccess || (e = alloc(&A2, (long)Rmax * 64)) != cudaSuccess ||
      (e = alloc(&Z, (long)Rmax * 64)) != cudaSuccess || (e = alloc(&B, (long)64 * Rmax)) != cudaSuccess ||
      (e = alloc(&Ch, 64 * 64 * 64)) != cudaSuccess || (e = alloc(&acc, 2)) != cudaSuccess ||
      (e = alloc(&eig, 3 * 64)) != cudaSuccess || (e = alloc(&Vh, 3 * 4096)) != cudaSuccess ||
      (e = alloc(&Mt, 64 * 64)) != cudaSuccess) {
    release();
    return cuda_error(P, e, "demag_recompress_tucker: workspace");
  }
  for (int p = 0; p < 3; ++p) {
    if ((e = alloc(&Y[p], (long)64 * n[p])) != cudaSuccess || (e = alloc(&Q[p], (long)64 * n[p])) != cudaSuccess) {
      release();
      return cuda_error(P, e, "demag_recompress_tucker: workspace");
    }
  }
#define RC_LAUNCH(name, ...)                                 \
  do {                                                       \
    DEMAG_LAUNCH(P, kFamMisc, st, __VA_ARGS__);              \
    if ((e = cudaGetLastError()) != cudaSuccess) {           \
      release();                                             \
      return cuda_error(P, e, name);                         \
    }                                                        \
  } while (0)
  // 1. factors in FP64, dense component cores
  {
    long boff = 0;
    for (int p = 0; p < 3; ++p) {
      const float* block = V + boff;
      for (int q = 0; q < 3; ++q)
        RC_LAUNCH("rc_gather_kernel", rc_gather_kernel<<<rc_blocks((long)Rr[p] * n[p]), 256, 0, st>>>(
                                          q, p, cv.rho[p], r[p], n[p], block, W + woff[q][p]));
      boff += 3L * cv.rho[p] * r[p] * n[p];
    }
    const long gsize = (long)r[0] * r[1] * r[2];
    const long csize = (long)cv.rho[0] * cv.rho[1] * cv.rho[2];
    for (int q = 0; q < 3; ++q)
      RC_LAUNCH("rc_core_kernel", rc_core_kernel<<<rc_blocks(Rtot), 256, 0, st>>>(
                                      cv.rho[0], cv.rho[1], cv.rho[2], r[0], r[1], r[2], cv.core + q * csize,
                                      core + q * gsize, E + q * Rtot));
  }
  // 2. ||phi||^2 = sum_{q,q'} <E_q, E_q' x_p (W_qp^T W_q'p)>
  DEMAG_CUDA(P, cudaMemsetAsync(acc, 0, sizeof(double) * 2, st));
  for (int q = 0; q < 3; ++q)
    for (int q2 = q; q2 < 3; ++q2) {
      const double* X = E + q2 * Rtot;
      double* outs[3] = {T1, T2, T1};
      for (int p = 0; p < 3; ++p) {
        RC_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)Rr[p] * Rr[p] * 32), 256, 0, st>>>(
                                        n[p], Rr[p], Rr[p], W + woff[q][p], W + woff[q2][p], G));
        RC_LAUNCH("rc_mode_kernel", rc_mode_kernel<<<rc_blocks(Rtot), 256, 0, st>>>(
                                        Rr[0], Rr[1], Rr[2], p, Rr[p], X, G, outs[p], 0));
        X = outs[p];
      }
      // the pair (q2, q) gives the same inner product: count it twice
      RC_LAUNCH("rc_dot_kernel", rc_dot_kernel<<<rc_blocks(Rtot), 256, 0, st>>>(Rtot, E + q * Rtot, X, acc));
      if (q2 != q) RC_LAUNCH("rc_dot_kernel", rc_dot_kernel<<<rc_blocks(Rtot), 256, 0, st>>>(Rtot, E + q * Rtot, X, acc));
    }
  double phi2 = 0.0;
  DEMAG_CUDA(P, cudaMemcpyAsync(&phi2, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  DEMAG_CUDA(P, cudaStreamSynchronize(st));
  if (!(phi2 > 0.0)) {
    release();
    return set_error(P, DEMAG_EINVAL, "demag_recompress_tucker: the potential is zero");
  }
  // 3. sketched ranges, growing the sample count until the projection error is below tol/2
  int kd[3] = {0, 0, 0};
  double es2 = 0.0;
  const unsigned long long seed = 0x5EEDull;
  for (int k = 16;; k *= 2) {
    for (int p = 0; p < 3; ++p) kd[p] = std::min(k, n[p]);
    for (int p = 0; p < 3; ++p) {
      const int s = (p + 1) % 3, rr = (p + 2) % 3;
      for (int q = 0; q < 3; ++q) {
        RC_LAUNCH("rc_probe_kernel", rc_probe_kernel<<<rc_blocks((long)Rr[s] * kd[p]), 256, 0, st>>>(
                                         n[s], Rr[s], kd[p], s, seed, W + woff[q][s], A1));
        RC_LAUNCH("rc_probe_kernel", rc_probe_kernel<<<rc_blocks((long)Rr[rr] * kd[p]), 256, 0, st>>>(
                                         n[rr], Rr[rr], kd[p], rr, seed, W + woff[q][rr], A2));
        RC_LAUNCH("rc_sketch_kernel", rc_sketch_kernel<<<rc_blocks((long)Rr[p] * kd[p]), 256, 0, st>>>(
                                          Rr[0], Rr[1], Rr[2], p, kd[p], E + q * Rtot, A1, A2, Z));
        RC_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)kd[p] * n[p]), 256, 0, st>>>(
                                         n[p], Rr[p], kd[p], W + woff[q][p], Z, Y[p], q > 0));
      }
      RC_LAUNCH("rc_qr_kernel", rc_qr_kernel<<<1, 256, 0, st>>>(kd[p], n[p], Y[p], Q[p], Rq));
    }
    // C = sum_q E_q x_p (Q_p^T W_qp)
    const long csz = (long)kd[0] * kd[1] * kd[2];
    for (int q = 0; q < 3; ++q) {
      const double* X = E + q * Rtot;
      int d[3] = {Rr[0], Rr[1], Rr[2]};
      double* outs[3] = {T1, T2, Ch};
      for (int p = 0; p < 3; ++p) {
        RC_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)kd[p] * Rr[p] * 32), 256, 0, st>>>(
                                        n[p], kd[p], Rr[p], Q[p], W + woff[q][p], B));
        const long osz = (long)(p == 0 ? kd[0] : d[0]) * (p == 1 ? kd[1] : d[1]) * (p == 2 ? kd[2] : d[2]);
        RC_LAUNCH("rc_mode_kernel", rc_mode_kernel<<<rc_blocks(osz), 256, 0, st>>>(
                                        d[0], d[1], d[2], p, kd[p], X, B, outs[p], p == 2 && q > 0));
        d[p] = kd[p];
        X = outs[p];
      }
    }
    DEMAG_CUDA(P, cudaMemsetAsync(acc + 1, 0, sizeof(double), st));
    RC_LAUNCH("rc_dot_kernel", rc_dot_kernel<<<rc_blocks(csz), 256, 0, st>>>(csz, Ch, Ch, acc + 1));
    double c2 = 0.0;
    DEMAG_CUDA(P, cudaMemcpyAsync(&c2, acc + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(P, cudaStreamSynchronize(st));
    es2 = std::max(0.0, phi2 - c2);
    const bool full = kd[0] == n[0] && kd[1] == n[1] && kd[2] == n[2];
    if (es2 <= 0.0625 * tol * tol * phi2 || full) break;
    if (k >= 64) {
      release();
      return set_error(P, DEMAG_EUNSUPPORTED,
                       "demag_recompress_tucker: ranks above 64 needed for tol %g (projection error %g)", tol,
                       sqrt(es2 / phi2));
    }
  }
  // 4. HOSVD of the small core, truncated within the remaining error budget
  const int npad = std::max(kd[0], std::max(kd[1], kd[2]));
  const int nev = npad + (npad & 1);
  {
    const size_t smem = sizeof(double) * 2 * nev * nev;
    static unsigned long long attr = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr & (1ull << (dev & 63)))) {
      DEMAG_CUDA(P, cudaFuncSetAttribute(rc_core_hosvd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         2 * 64 * 64 * 8));
      attr |= 1ull << (dev & 63);
    }
    RC_LAUNCH("rc_core_hosvd_kernel",
              rc_core_hosvd_kernel<<<1, 256, smem, st>>>(kd[0], kd[1], kd[2], nev, Ch, eig, Vh));
  }
  std::vector<double> eh(3 * 64), vh(3 * 4096);
  DEMAG_CUDA(P, cudaMemcpyAsync(eh.data(), eig, sizeof(double) * 3 * 64, cudaMemcpyDeviceToHost, st));
  DEMAG_CUDA(P, cudaMemcpyAsync(vh.data(), Vh, sizeof(double) * 3 * 4096, cudaMemcpyDeviceToHost, st));
  DEMAG_CUDA(P, cudaStreamSynchronize(st));
  const double budget = std::max(0.0, tol * tol * phi2 - es2);
  double tails = 0.0;
  int rk[3];
  for (int p = 0; p < 3; ++p) {
    double tot = 0.0;
    for (int i = 0; i < kd[p]; ++i) tot += std::max(0.0, eh[64 * p + i]);
    double tail = tot;
    rk[p] = kd[p];
    for (int rr = 1; rr <= kd[p]; ++rr) {
      tail -= std::max(0.0, eh[64 * p + rr - 1]);
      if (tail <= budget / 3.0) {
        rk[p] = rr;
        break;
      }
    }
    double kept = 0.0;
    for (int i = 0; i < rk[p]; ++i) kept += std::max(0.0, eh[64 * p + i]);
    tails += std::max(0.0, tot - kept);
  }
  // 5. U_p = Q_p V_p[:, :rk] (rows of U_out), C' = C x_p V_p[:, :rk]^T
  {
    long uoff = 0;
    for (int p = 0; p < 3; ++p) {
      std::vector<double> vp((size_t)kd[p] * kd[p]);
      for (int c = 0; c < kd[p]; ++c)
        for (int i = 0; i < kd[p]; ++i) vp[(size_t)c * kd[p] + i] = vh[4096 * p + (size_t)c * kd[p] + i];
      DEMAG_CUDA(P, cudaMemcpyAsync(Mt, vp.data(), sizeof(double) * vp.size(), cudaMemcpyHostToDevice, st));
      RC_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)kd[p] * n[p]), 256, 0, st>>>(
                                       n[p], kd[p], kd[p], Q[p], Mt, Y[p], 0));
      DEMAG_CUDA(P, cudaStreamSynchronize(st));  // Mt is reused
      // rows 0..rk-1 of Y[p] ([k][n] column-major) are the columns of U_p
      std::vector<float> tmp;
      std::vector<double> yh((size_t)rk[p] * n[p]);
      DEMAG_CUDA(P, cudaMemcpy(yh.data(), Y[p], sizeof(double) * yh.size(), cudaMemcpyDeviceToHost));
      tmp.resize(yh.size());
      for (size_t i = 0; i < yh.size(); ++i) tmp[i] = (float)yh[i];
      DEMAG_CUDA(P, cudaMemcpy(U_out + uoff, tmp.data(), sizeof(float) * tmp.size(), cudaMemcpyHostToDevice));
      uoff += (long)rk[p] * n[p];
    }
    double* X = Ch;
    int d[3] = {kd[0], kd[1], kd[2]};
    double* outs[3] = {T1, T2, T1};  // T1 is free again once mode 2 has read it
    for (int p = 0; p < 3; ++p) {
      std::vector<double> mt((size_t)rk[p] * kd[p]);  // [a][b] = V_p[b][a]
      for (int a = 0; a < rk[p]; ++a)
        for (int b = 0; b < kd[p]; ++b) mt[(size_t)a * kd[p] + b] = vh[4096 * p + (size_t)b * kd[p] + a];
      DEMAG_CUDA(P, cudaMemcpy(Mt, mt.data(), sizeof(double) * mt.size(), cudaMemcpyHostToDevice));
      const long osz = (long)(p == 0 ? rk[0] : d[0]) * (p == 1 ? rk[1] : d[1]) * (p == 2 ? rk[2] : d[2]);
      RC_LAUNCH("rc_mode_kernel", rc_mode_kernel<<<rc_blocks(osz), 256, 0, st>>>(d[0], d[1], d[2], p, rk[p], X, Mt,
                                                                                 outs[p], 0));
      DEMAG_CUDA(P, cudaStreamSynchronize(st));
      d[p] = rk[p];
      X = outs[p];
    }
    const long cn = (long)rk[0] * rk[1] * rk[2];
    std::vector<double> ch(cn);
    DEMAG_CUDA(P, cudaMemcpy(ch.data(), X, sizeof(double) * cn, cudaMemcpyDeviceToHost));
    std::vector<float> cf(cn);
    for (long i = 0; i < cn; ++i) cf[i] = (float)ch[i];
    DEMAG_CUDA(P, cudaMemcpy(core_out, cf.data(), sizeof(float) * cn, cudaMemcpyHostToDevice));
  }
#undef RC_LAUNCH
  release();
  for (int p = 0; p < 3; ++p) ranks_out[p] = rk[p];
  if (err_out) *err_out = sqrt((es2 + tails) / phi2);
  return DEMAG_OK;
}

// smallest r >= 1 whose discarded eigenvalues (descending, k of them) sum to <= bound; tail returned
static int tail_rank(const double* ev, int k, double bound, double* tail_out) {
  double tot = 0.0;
  for (int i = 0; i < k; ++i) tot += std::max(0.0, ev[i]);
  double tail = tot;
  int r = k;
  for (int rr = 1; rr <= k; ++rr) {
    tail -= std::max(0.0, ev[rr - 1]);
    if (tail <= bound) {
      r = rr;
      break;
    }
  }
  double kept = 0.0;
  for (int i = 0; i < r; ++i) kept += std::max(0.0, ev[i]);
  *tail_out = std::max(0.0, tot - kept);
  return r;
}

extern "C" demag_status demag_round_tt(demag_plan* P, const int r[2], const float* w, const float* G1,
                                       const float* G2, const float* G3, double tol, int ranks_out[2],
                                       float* G1_out, float* G2_out, float* G3_out, double* err_out,
                                       void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_round_tt: plan is NULL");
  if (!r || !w || !G1 || !G2 || !G3 || !ranks_out || !G1_out || !G2_out || !G3_out)
    return set_error(P, DEMAG_EINVAL, "demag_round_tt: NULL pointer");
  if (r[0] < 1 || r[1] < 1) return set_error(P, DEMAG_EINVAL, "demag_round_tt: ranks must be >= 1");
  if (!(tol > 0.0 && tol < 1.0)) return set_error(P, DEMAG_EINVAL, "demag_round_tt: tol must be in (0, 1)");
  cudaStream_t st = (cudaStream_t)stream;
  const int T = 3 * P->M, ra = r[0], rb = r[1];
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const long nA = (long)T * ra * n1, nB = (long)T * ra * rb * n2, nC = (long)T * rb * n3;
  const long kmax = 64;
  std::vector<void*> owned;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** ptr, long count) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(ptr, sizeof(double) * (size_t)std::max(count, 1L));
    if (e == cudaSuccess) owned.push_back(*ptr);
  };
  auto release = [&]() {
    for (void* q : owned) cudaFree(q);
    owned.clear();
  };
  double *wd, *A, *B, *C, *GA, *GB, *GC, *acc, *CW1, *CW2, *BW, *hh, *Y1, *Q1, *R1, *AP, *F, *Y2, *Q2, *R2, *wE, *Z;
  double *ZZ, *VZ, *M1, *ev, *EV, *Wm, *Vp, *Qv, *Rv, *Zp, *O1, *O2, *O3;
  const long m12 = kmax * n2;  // rows of the (1,2) unfolding at most
  alloc(&wd, T);
  alloc(&A, nA);
  alloc(&B, nB);
  alloc(&C, nC);
  alloc(&GA, (long)T * ra * T * ra);
  alloc(&GB, (long)T * ra * rb * T * ra * rb);
  alloc(&GC, (long)T * rb * T * rb);
  alloc(&acc, 2);
  alloc(&CW1, (long)T * rb * kmax);
  alloc(&CW2, (long)T * rb * kmax);
  alloc(&BW, (long)T * ra * rb * kmax);
  alloc(&hh, (long)T * ra * kmax);
  alloc(&Y1, kmax * n1);
  alloc(&Q1, kmax * n1);
  alloc(&R1, kmax * kmax);
  alloc(&AP, kmax * T * ra);
  alloc(&F, (long)T * ra * n2 * kmax);
  alloc(&Y2, kmax * m12);
  alloc(&Q2, kmax * m12);
  alloc(&R2, kmax * kmax);
  alloc(&wE, (long)T * rb * kmax);
  alloc(&Z, kmax * n3);
  alloc(&ZZ, kmax * kmax);
  alloc(&VZ, kmax * m12);
  alloc(&M1, kmax * kmax);
  alloc(&ev, kmax);
  alloc(&EV, kmax * kmax);
  alloc(&Wm, kmax * kmax);
  alloc(&Vp, kmax * m12);
  alloc(&Qv, kmax * m12);
  alloc(&Rv, kmax * kmax);
  alloc(&Zp, kmax * n3);
  alloc(&O1, kmax * n1);
  alloc(&O2, kmax * m12);
  alloc(&O3, kmax * n3);
  if (e != cudaSuccess) {
    release();
    return cuda_error(P, e, "demag_round_tt: workspace");
  }
#define TT_LAUNCH(name, ...)                                 \
  do {                                                       \
    DEMAG_LAUNCH(P, kFamMisc, st, __VA_ARGS__);              \
    if ((e = cudaGetLastError()) != cudaSuccess) {           \
      release();                                             \
      return cuda_error(P, e, name);                         \
    }                                                        \
  } while (0)
#define TT_CUDA(call)                                        \
  do {                                                       \
    if ((e = (call)) != cudaSuccess) {                       \
      release();                                             \
      return cuda_error(P, e, #call);                        \
    }                                                        \
  } while (0)
  TT_LAUNCH("rc_f2d_kernel", rc_f2d_kernel<<<rc_blocks(T), 256, 0, st>>>(T, w, wd));
  TT_LAUNCH("rc_f2d_kernel", rc_f2d_kernel<<<rc_blocks(nA), 256, 0, st>>>(nA, G1, A));
  TT_LAUNCH("rc_f2d_kernel", rc_f2d_kernel<<<rc_blocks(nB), 256, 0, st>>>(nB, G2, B));
  TT_LAUNCH("rc_f2d_kernel", rc_f2d_kernel<<<rc_blocks(nC), 256, 0, st>>>(nC, G3, C));
  // 1. ||phi||^2 from the pairwise Grams of the terms
  const long na = (long)T * ra, nbb = (long)T * ra * rb, nc = (long)T * rb;
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks(na * na * 32), 256, 0, st>>>(n1, (int)na, (int)na, A, A, GA));
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks(nbb * nbb * 32), 256, 0, st>>>(n2, (int)nbb, (int)nbb, B, B, GB));
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks(nc * nc * 32), 256, 0, st>>>(n3, (int)nc, (int)nc, C, C, GC));
  TT_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 2, st));
  TT_LAUNCH("tt_norm_kernel", tt_norm_kernel<<<rc_blocks((long)T * T), 256, 0, st>>>(T, ra, rb, wd, GA, GB, GC, acc));
  double phi2 = 0.0;
  TT_CUDA(cudaMemcpyAsync(&phi2, acc, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  if (!(phi2 > 0.0)) {
    release();
    return set_error(P, DEMAG_EINVAL, "demag_round_tt: the potential is zero");
  }
  // 2. sketched ranges
  const unsigned long long seed = 0x7717ull;
  int k1 = 0, k2 = 0;
  double es2 = 0.0;
  for (int k = 16;; k *= 2) {
    k1 = std::min(k, n1);
    k2 = (int)std::min<long>(std::min<long>(k, (long)k1 * n2), n3);
    TT_LAUNCH("rc_probe_kernel", rc_probe_kernel<<<rc_blocks(nc * k1), 256, 0, st>>>(n3, (int)nc, k1, 2, seed, C, CW1));
    TT_LAUNCH("rc_probe_kernel", rc_probe_kernel<<<rc_blocks(nbb * k1), 256, 0, st>>>(n2, (int)nbb, k1, 1, seed, B, BW));
    TT_LAUNCH("tt_h_kernel", tt_h_kernel<<<rc_blocks(na * k1), 256, 0, st>>>(T, ra, rb, k1, wd, BW, CW1, hh));
    TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)k1 * n1), 256, 0, st>>>(n1, (int)na, k1, A, hh, Y1, 0));
    TT_LAUNCH("rc_qr_kernel", rc_qr_kernel<<<1, 256, 0, st>>>(k1, n1, Y1, Q1, R1));
    TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)k1 * na * 32), 256, 0, st>>>(n1, k1, (int)na, Q1, A, AP));
    TT_LAUNCH("rc_probe_kernel", rc_probe_kernel<<<rc_blocks(nc * k2), 256, 0, st>>>(n3, (int)nc, k2, 3, seed, C, CW2));
    TT_LAUNCH("tt_f_kernel", tt_f_kernel<<<rc_blocks(na * n2 * k2), 256, 0, st>>>(T, ra, rb, n2, k2, wd, B, CW2, F));
    TT_LAUNCH("tt_y2_kernel", tt_y2_kernel<<<rc_blocks((long)k1 * n2 * k2), 256, 0, st>>>(k1, n2, k2, (int)na, AP, F, Y2));
    TT_LAUNCH("rc_qr_kernel", rc_qr_kernel<<<1, 256, 0, st>>>(k2, k1 * n2, Y2, Q2, R2));
    TT_LAUNCH("tt_p_kernel", tt_p_kernel<<<rc_blocks(na * n2 * k2), 256, 0, st>>>(k1, n2, k2, (int)na, Q2, AP, F));
    TT_LAUNCH("tt_e_kernel", tt_e_kernel<<<rc_blocks(nc * k2), 256, 0, st>>>(T, ra, rb, n2, k2, wd, F, B, wE));
    TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)k2 * n3), 256, 0, st>>>(n3, (int)nc, k2, C, wE, Z, 0));
    TT_CUDA(cudaMemsetAsync(acc + 1, 0, sizeof(double), st));
    TT_LAUNCH("rc_dot_kernel", rc_dot_kernel<<<rc_blocks((long)k2 * n3), 256, 0, st>>>((long)k2 * n3, Z, Z, acc + 1));
    double z2 = 0.0;
    TT_CUDA(cudaMemcpyAsync(&z2, acc + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaStreamSynchronize(st));
    es2 = std::max(0.0, phi2 - z2);
    const bool full = k1 == n1 && k2 == (int)std::min<long>((long)k1 * n2, n3);
    if (es2 <= 0.0625 * tol * tol * phi2 || full) break;
    if (k >= 64) {
      release();
      return set_error(P, DEMAG_EUNSUPPORTED, "demag_round_tt: ranks above 64 needed for tol %g (projection error %g)",
                       tol, sqrt(es2 / phi2));
    }
  }
  // 3. truncations of the projected train: ||phi - phi_hat|| <= sqrt(es2) + sqrt(tail1 + tail2),
  // so the two tails share (tol ||phi|| - sqrt(es2))^2, half each
  const double room = std::max(0.0, tol * sqrt(phi2) - sqrt(es2));
  const double half = 0.5 * room * room;
  auto eig = [&](int k, const double* S, std::vector<double>& evh, std::vector<double>& vh) -> demag_status {
    const int n = k + (k & 1);
    TT_LAUNCH("rc_eig_kernel", rc_eig_kernel<<<1, 256, sizeof(double) * 2 * n * n, st>>>(k, n, S, ev, EV));
    evh.resize(k);
    vh.resize((size_t)k * k);
    TT_CUDA(cudaMemcpyAsync(evh.data(), ev, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaMemcpyAsync(vh.data(), EV, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaStreamSynchronize(st));
    return DEMAG_OK;
  };
  {
    static unsigned long long attr = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr & (1ull << (dev & 63)))) {
      TT_CUDA(cudaFuncSetAttribute(rc_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * 64 * 64 * 8));
      attr |= 1ull << (dev & 63);
    }
  }
  std::vector<double> evh, vh;
  // mode 1
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)k2 * k2 * 32), 256, 0, st>>>(n3, k2, k2, Z, Z, ZZ));
  TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)k2 * k1 * n2), 256, 0, st>>>(k1 * n2, k2, k2, Q2, ZZ, VZ, 0));
  TT_LAUNCH("tt_m1_kernel", tt_m1_kernel<<<rc_blocks((long)k1 * k1 * 32), 256, 0, st>>>(k1, n2, k2, Q2, VZ, M1));
  demag_status rs = eig(k1, M1, evh, vh);
  if (rs != DEMAG_OK) return rs;
  double tail1 = 0.0, tail2 = 0.0;
  const int q1 = tail_rank(evh.data(), k1, half, &tail1);
  std::vector<double> w1((size_t)k1 * q1);  // [a][i]
  for (int a = 0; a < k1; ++a)
    for (int i = 0; i < q1; ++i) w1[(size_t)a * q1 + i] = vh[(size_t)a * k1 + i];
  TT_CUDA(cudaMemcpyAsync(Wm, w1.data(), sizeof(double) * w1.size(), cudaMemcpyHostToDevice, st));
  TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)q1 * n1), 256, 0, st>>>(n1, k1, q1, Q1, Wm, O1, 0));
  TT_LAUNCH("tt_vprime_kernel", tt_vprime_kernel<<<rc_blocks((long)q1 * n2 * k2), 256, 0, st>>>(k1, q1, n2, k2, Wm, Q2, Vp));
  TT_LAUNCH("rc_qr_kernel", rc_qr_kernel<<<1, 256, 0, st>>>(k2, q1 * n2, Vp, Qv, Rv));
  std::vector<double> rvh((size_t)k2 * k2), rvt((size_t)k2 * k2);
  TT_CUDA(cudaMemcpyAsync(rvh.data(), Rv, sizeof(double) * rvh.size(), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  for (int j = 0; j < k2; ++j)
    for (int c = 0; c < k2; ++c) rvt[(size_t)c * k2 + j] = rvh[(size_t)j * k2 + c];  // Zm[c][j] = Rv[j][c]
  TT_CUDA(cudaMemcpyAsync(Wm, rvt.data(), sizeof(double) * rvt.size(), cudaMemcpyHostToDevice, st));
  TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)k2 * n3), 256, 0, st>>>(n3, k2, k2, Z, Wm, Zp, 0));
  // mode 2 (the (1,2) interface)
  TT_CUDA(cudaStreamSynchronize(st));
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)k2 * k2 * 32), 256, 0, st>>>(n3, k2, k2, Zp, Zp, ZZ));
  rs = eig(k2, ZZ, evh, vh);
  if (rs != DEMAG_OK) return rs;
  const int q2 = tail_rank(evh.data(), k2, half, &tail2);
  std::vector<double> w2((size_t)k2 * q2);
  for (int j = 0; j < k2; ++j)
    for (int c = 0; c < q2; ++c) w2[(size_t)j * q2 + c] = vh[(size_t)j * k2 + c];
  TT_CUDA(cudaMemcpyAsync(Wm, w2.data(), sizeof(double) * w2.size(), cudaMemcpyHostToDevice, st));
  TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)q2 * q1 * n2), 256, 0, st>>>(q1 * n2, k2, q2, Qv, Wm, O2, 0));
  // 4. last core as the orthogonal projection of phi itself on the first two cores,
  // G3 = G2^T (G1^T phi); then ||phi - phi_hat||^2 = ||phi||^2 - ||G3||^2 exactly
  TT_LAUNCH("rc_gram_kernel", rc_gram_kernel<<<rc_blocks((long)q1 * na * 32), 256, 0, st>>>(n1, q1, (int)na, O1, A, AP));
  TT_LAUNCH("tt_p_kernel", tt_p_kernel<<<rc_blocks(na * n2 * q2), 256, 0, st>>>(q1, n2, q2, (int)na, O2, AP, F));
  TT_LAUNCH("tt_e_kernel", tt_e_kernel<<<rc_blocks(nc * q2), 256, 0, st>>>(T, ra, rb, n2, q2, wd, F, B, wE));
  TT_LAUNCH("rc_range_kernel", rc_range_kernel<<<rc_blocks((long)q2 * n3), 256, 0, st>>>(n3, (int)nc, q2, C, wE, O3, 0));
  TT_CUDA(cudaMemsetAsync(acc + 1, 0, sizeof(double), st));
  TT_LAUNCH("rc_dot_kernel", rc_dot_kernel<<<rc_blocks((long)q2 * n3), 256, 0, st>>>((long)q2 * n3, O3, O3, acc + 1));
  double g32 = 0.0;
  TT_CUDA(cudaMemcpyAsync(&g32, acc + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CUDA(cudaStreamSynchronize(st));
  // outputs (FP32): G1 [q1][n1]; G2 [(b c)][n2] from O2 [c][(b i2)]; G3 [q2][n3]
  {
    std::vector<double> o1((size_t)q1 * n1), o2((size_t)q2 * q1 * n2), o3((size_t)q2 * n3);
    TT_CUDA(cudaMemcpyAsync(o1.data(), O1, sizeof(double) * o1.size(), cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaMemcpyAsync(o2.data(), O2, sizeof(double) * o2.size(), cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaMemcpyAsync(o3.data(), O3, sizeof(double) * o3.size(), cudaMemcpyDeviceToHost, st));
    TT_CUDA(cudaStreamSynchronize(st));
    std::vector<float> f1(o1.begin(), o1.end()), f3(o3.begin(), o3.end()), f2((size_t)q1 * q2 * n2);
    for (int b = 0; b < q1; ++b)
      for (int c = 0; c < q2; ++c)
        for (int i2 = 0; i2 < n2; ++i2)
          f2[((size_t)b * q2 + c) * n2 + i2] = (float)o2[(size_t)c * q1 * n2 + (size_t)b * n2 + i2];
    TT_CUDA(cudaMemcpyAsync(G1_out, f1.data(), sizeof(float) * f1.size(), cudaMemcpyHostToDevice, st));
    TT_CUDA(cudaMemcpyAsync(G2_out, f2.data(), sizeof(float) * f2.size(), cudaMemcpyHostToDevice, st));
    TT_CUDA(cudaMemcpyAsync(G3_out, f3.data(), sizeof(float) * f3.size(), cudaMemcpyHostToDevice, st));
    TT_CUDA(cudaStreamSynchronize(st));
  }
#undef TT_LAUNCH
#undef TT_CUDA
  release();
  ranks_out[0] = q1;
  ranks_out[1] = q2;
  if (err_out) *err_out = sqrt(std::max(0.0, phi2 - g32) / phi2);
  return DEMAG_OK;
}
