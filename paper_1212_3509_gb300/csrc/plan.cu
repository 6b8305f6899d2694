// Plan setup: sinc nodes, FP64 Toeplitz generators, circulant symbols.
//
// Sec. 3.4 (Eq. gauss_trans, Lemma 2, Cor. 3 Eq. kron_operator), Eq. f_anal
// (erf / exp differences), Sec. 4.2 (Eq. conv_op, conv_pot, fft_pot).
#include <cstdarg>
#include <cmath>
#include <atomic>
#include <new>
#include <vector>

#include "internal.h"
#include "fft.cuh"

namespace demag {

static thread_local char g_err[512] = "no error";

demag_status set_error(demag_plan* plan, demag_status st, const char* fmt, ...) {
  char* dst = plan ? plan->err : g_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
  if (plan) snprintf(g_err, sizeof(g_err), "%s", plan->err);
  return st;
}

demag_status cuda_error(demag_plan* plan, cudaError_t e, const char* where) {
  demag_status st = (e == cudaErrorMemoryAllocation) ? DEMAG_ENOMEM : DEMAG_ECUDA;
  return set_error(plan, st, "%s: %s", where, cudaGetErrorString(e));
}

void prof_begin(demag_plan* P, int family, cudaStream_t st) {
  if (!P || !P->prof_on) return;
  while (P->prof_used + 2 > P->prof_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { P->prof_on = false; return; }
    P->prof_pool.push_back(e);
  }
  demag_plan::ProfRec r;
  r.family = family;
  r.a = P->prof_pool[P->prof_used++];
  r.b = P->prof_pool[P->prof_used++];
  cudaEventRecord(r.a, st);
  P->prof.push_back(r);
}

void prof_end(demag_plan* P, cudaStream_t st) {
  if (!P || !P->prof_on || P->prof.empty()) return;
  cudaEventRecord(P->prof.back().b, st);
}

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// ---------------------------------------------------------------- kernels

// t_k = k theta, tau_k = sinh t_k, omega_k = 2 theta cosh t_k sinh^2 t_k,
// theta = c0 ln(M) / M (Cor. 3 with the folded symmetric rule).
__global__ void nodes_kernel(int M, double c0, double cscale, double* nodes, double* scale) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double theta = c0 * log((double)M) / (double)M;
  double t = theta * (double)(k + 1);
  double tau = sinh(t);
  double omega = 2.0 * theta * cosh(t) * tau * tau;
  nodes[k] = t;
  nodes[M + k] = tau;
  nodes[2 * M + k] = omega;
  scale[k] = cscale * omega;
}

// E_k^(p)[d] and F_k^(p)[d] of Eq. f_anal for d = -(n_p-1)..n_p-1, FP64.
// E, d != 0, uses erf(tau b) - erf(tau a) while tau a < 1/2 and otherwise
// the tail form exp(-tau^2 a^2) (erfcx(tau a) - exp(-tau^2 (b^2-a^2)) erfcx(tau b)),
// which is the same difference without cancellation at large tau.
// F uses exp(-tau^2 a^2) * (-expm1(-2 |d| tau^2 hh^2)) / (2 tau^2).
__global__ void generators_kernel(int M, int glen, GridInfo g, const double* nodes, double* gen) {
  const long total = (long)M * 2 * 3 * glen;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    int e = (int)(idx % glen);
    long rest = idx / glen;
    int p = (int)(rest % 3);
    rest /= 3;
    int type = (int)(rest % 2);
    int k = (int)(rest / 2);
    int n = g.n[p];
    double val = 0.0;
    if (e < 2 * n - 1) {
      int d = e - (n - 1);
      int ad = d < 0 ? -d : d;
      double tau = nodes[M + k];
      double hh = g.hh[p];
      double a = ((double)ad - 0.5) * hh;
      double b = a + hh;
      if (type == 0) {
        const double sqrt_pi = 1.7724538509055160273;
        if (ad == 0) {
          val = sqrt_pi / tau * erf(0.5 * tau * hh);
        } else {
          double ta = tau * a, tb = tau * b;
          double diff;
          if (ta < 0.5) {
            diff = erf(tb) - erf(ta);
          } else {
            diff = exp(-ta * ta) * (erfcx(ta) - exp(-2.0 * ad * tau * tau * hh * hh) * erfcx(tb));
          }
          val = 0.5 * sqrt_pi / tau * diff;
        }
      } else if (ad != 0) {
        double t2 = tau * tau;
        double mag = exp(-t2 * a * a) * (-expm1(-2.0 * ad * t2 * hh * hh)) / (2.0 * t2);
        val = d > 0 ? mag : -mag;
      }
    }
    gen[idx] = val;
  }
}

struct TwiddleD {
  int N;
  __device__ double2 operator()(int m) const {
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    return make_double2(c, s);
  }
};

// Circulant symbol of one generator (Sec. 4.2, Eq. fft_pot): c[j] = t[j],
// c[L-d] = t[-d], zero elsewhere; real FFT of length L = 2N in FP64; E keeps
// Re/L and F keeps Im/L (E even -> real symbol, F odd -> imaginary symbol).
// Generators are rows (k * nsets + set) * 3 + axis of `gen`; with nsets = 2
// the set is the type (0 E, 1 F), with nsets = 3 it is the component q of a
// compressed kernel, whose axis-q generators are odd (F-like).
template <int LOGN>
__global__ void __launch_bounds__(256) symbol_kernel(int M, int nsets, int glen, int axis, int n, int symstride,
                                                     const double* gen, float* sym) {
  constexpr int N = 1 << LOGN;
  constexpr int L = 2 * N;
  extern __shared__ double2 zs[];
  const int k = blockIdx.x, set = blockIdx.y;
  const int type = nsets == 2 ? set : (set == axis ? 1 : 0);
  const double* t = gen + (((long)k * nsets + set) * 3 + axis) * glen;  // t[d + n - 1]
  auto circ = [&](int j) -> double {
    if (j < n) return t[j + n - 1];
    if (j > L - n) return t[(j - L) + n - 1];
    return 0.0;
  };
  for (int j = threadIdx.x; j < N; j += blockDim.x) zs[j] = make_double2(circ(2 * j), circ(2 * j + 1));
  __syncthreads();
  fft_inplace<LOGN, 256, false>(zs, threadIdx.x, TwiddleD{N});
  float* out = sym + (((long)k * nsets + set) * 3 + axis) * symstride;
  for (int f = threadIdx.x; f <= N; f += blockDim.x) {
    double2 a = zs[f % N];
    double2 b = zs[(N - f) % N];
    // C[f] = (A + conj B)/2 - i/2 e^{-2 pi i f / L} (A - conj B)
    double ex = 0.5 * (a.x + b.x), ey = 0.5 * (a.y - b.y);
    double dx = 0.5 * (a.x - b.x), dy = 0.5 * (a.y + b.y);
    double s, c;
    sincospi(-2.0 * (double)f / (double)L, &s, &c);
    // w*d with w = (c, s): (c dx - s dy, c dy + s dx); times -i: (im, -re)
    double wx = c * dx - s * dy, wy = c * dy + s * dx;
    double Cx = ex + wy, Cy = ey - wx;
    out[f] = (float)((type == 0 ? Cx : Cy) / (double)L);
  }
}

// (s[f], s[N - f]) pairs of one axis for the structured kernels, f < N = L_p/2
__global__ void sympair_kernel(int M, int nsets, int axis, int N, int symstride, int pairstride, const float* sym,
                               float2* pair) {
  const long total = (long)M * nsets * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const int f = (int)(i % N);
    const long kt = i / N;  // k * nsets + set
    const float* s = sym + (kt * 3 + axis) * symstride;
    pair[(kt * 3 + axis) * pairstride + f] = make_float2(s[f], s[N - f]);
  }
}

__global__ void twiddle_kernel(int L, float2* tw) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= L) return;
  double s, c;
  sincospi(-2.0 * (double)m / (double)L, &s, &c);
  tw[m] = make_float2((float)c, (float)s);
}

template <int LOGN>
static void launch_symbol(demag_plan* P, int axis, int M, int nsets, const double* gen, float* sym,
                          cudaStream_t st) {
  size_t smem = sizeof(double2) << LOGN;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(symbol_kernel<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  DEMAG_LAUNCH(P, kFamSetup, st,
               symbol_kernel<LOGN><<<dim3(M, nsets), 256, smem, st>>>(M, nsets, P->glen, axis, P->n[axis],
                                                                      P->Lmax / 2 + 1, gen, sym));
}

// Symbols of axis `axis` for generator rows [M][nsets][3][glen] into [M][nsets][3][Lmax/2 + 1].
void dispatch_symbol(demag_plan* P, int axis, int M, int nsets, const double* gen, float* sym, cudaStream_t st) {
  switch (ilog2(P->L[axis] / 2)) {
    case 0: launch_symbol<0>(P, axis, M, nsets, gen, sym, st); break;
    case 1: launch_symbol<1>(P, axis, M, nsets, gen, sym, st); break;
    case 2: launch_symbol<2>(P, axis, M, nsets, gen, sym, st); break;
    case 3: launch_symbol<3>(P, axis, M, nsets, gen, sym, st); break;
    case 4: launch_symbol<4>(P, axis, M, nsets, gen, sym, st); break;
    case 5: launch_symbol<5>(P, axis, M, nsets, gen, sym, st); break;
    case 6: launch_symbol<6>(P, axis, M, nsets, gen, sym, st); break;
    case 7: launch_symbol<7>(P, axis, M, nsets, gen, sym, st); break;
    case 8: launch_symbol<8>(P, axis, M, nsets, gen, sym, st); break;
    case 9: launch_symbol<9>(P, axis, M, nsets, gen, sym, st); break;
    case 10: launch_symbol<10>(P, axis, M, nsets, gen, sym, st); break;
    case 11: launch_symbol<11>(P, axis, M, nsets, gen, sym, st); break;
    case 12: launch_symbol<12>(P, axis, M, nsets, gen, sym, st); break;
    case 13: launch_symbol<13>(P, axis, M, nsets, gen, sym, st); break;
    default: break;
  }
}

}  // namespace demag

using namespace demag;

// ---------------------------------------------------------------- ABI

static std::atomic<unsigned long long> g_next_serial{1};  // plan serials (cache keys)

static void free_plan_buffers(demag_plan* P) {
  cudaFree(P->nodes);
  cudaFree(P->gen64);
  cudaFree(P->sym);
  cudaFree(P->sympair);
  cudaFree(P->scale);
  for (int p = 0; p < 3; ++p) {
    bool dup = false;
    for (int q = 0; q < p; ++q) dup |= (P->twid[q] == P->twid[p]);
    if (!dup) cudaFree(P->twid[p]);
  }
  cudaFree(P->T32);
  cudaFree(P->T64);
  cudaFree(P->fac64);
  cudaFree(P->T32t);
  cudaFree(P->T64t);
  cudaFree(P->T32d);
  cudaFree(P->T64d);
  cudaFree(P->gend);
  cudaFree(P->fib_ws);
  P->fib_ws = nullptr;
  for (auto& w : P->ws) cudaFree(w.base);
  cudaFree(P->dev_status);
  for (auto e : P->prof_pool) cudaEventDestroy(e);
  P->prof_pool.clear();
  tc_destroy(P);
  fft3d_destroy(P);
  compress_destroy(P);
  energy_destroy(P);
}

extern "C" demag_status demag_build_factors(const demag_grid_desc* d, demag_plan** out, void* stream) {
  if (!out) return set_error(nullptr, DEMAG_EINVAL, "demag_build_factors: out is NULL");
  *out = nullptr;
  if (!d) return set_error(nullptr, DEMAG_EINVAL, "demag_build_factors: desc is NULL");
  for (int p = 0; p < 3; ++p) {
    if (d->n[p] < 1) return set_error(nullptr, DEMAG_EINVAL, "n[%d] = %d must be >= 1", p, d->n[p]);
    if (!(d->h[p] > 0.0) || !std::isfinite(d->h[p]))
      return set_error(nullptr, DEMAG_EINVAL, "h[%d] must be positive and finite", p);
    if (d->n[p] > (1 << 20)) return set_error(nullptr, DEMAG_EUNSUPPORTED, "n[%d] too large", p);
  }
  if (d->R < 5 || d->R % 2 == 0)
    return set_error(nullptr, DEMAG_EINVAL, "R = %d must be odd and >= 5 (R = 2M+1)", d->R);
  if ((d->R - 1) / 2 > kMaxTerms)
    return set_error(nullptr, DEMAG_EUNSUPPORTED, "R = %d exceeds 2*%d+1", d->R, kMaxTerms);
  if (!(d->c0 > 0.0) || !std::isfinite(d->c0))
    return set_error(nullptr, DEMAG_EINVAL, "c0 must be positive and finite");

  cudaStream_t st = (cudaStream_t)stream;
  demag_plan* P = new (std::nothrow) demag_plan();
  if (!P) return set_error(nullptr, DEMAG_ENOMEM, "host allocation failed");
  snprintf(P->err, sizeof(P->err), "no error");
  P->serial = g_next_serial.fetch_add(1);
  P->R = d->R;
  P->M = (d->R - 1) / 2;
  P->c0 = d->c0;
  P->s = 0.0;
  P->nmax = 0;
  P->Lmax = 0;
  for (int p = 0; p < 3; ++p) {
    P->n[p] = d->n[p];
    P->h[p] = d->h[p];
    P->s = fmax(P->s, (double)d->n[p] * d->h[p]);
    P->nmax = P->n[p] > P->nmax ? P->n[p] : P->nmax;
  }
  for (int p = 0; p < 3; ++p) {
    P->hh[p] = P->h[p] / P->s;
    int L = next_pow2(2 * P->n[p] - 1);
    P->L[p] = L < 2 ? 2 : L;
    P->Lmax = P->L[p] > P->Lmax ? P->L[p] : P->Lmax;
  }
  P->glen = 2 * P->nmax - 1;
  P->tgroup = 0;
  for (int p = 0; p < 3; ++p) {
    P->toff[p] = P->tgroup;
    P->tgroup += (size_t)P->n[p] * P->n[p];
  }
  const int M = P->M;
  const bool fft_ok = P->Lmax / 2 <= (1 << kMaxFFTLog);

  auto fail = [&](demag_status s) {
    snprintf(g_err, sizeof(g_err), "%s", P->err);
    free_plan_buffers(P);
    delete P;
    return s;
  };
#define TRY_CUDA(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fail(cuda_error(P, e_, #call)); \
  } while (0)

  TRY_CUDA(cudaMalloc(&P->nodes, sizeof(double) * 3 * M));
  TRY_CUDA(cudaMalloc(&P->scale, sizeof(double) * M));
  TRY_CUDA(cudaMalloc(&P->gen64, sizeof(double) * (size_t)M * 6 * P->glen));
  TRY_CUDA(cudaMalloc(&P->dev_status, sizeof(int)));
  TRY_CUDA(cudaMemsetAsync(P->dev_status, 0, sizeof(int), st));

  DEMAG_LAUNCH(P, kFamSetup, st, nodes_kernel<<<(M + 63) / 64, 64, 0, st>>>(M, P->c0, kCPot * P->s, P->nodes, P->scale));
  TRY_CUDA(cudaGetLastError());
  GridInfo g;
  for (int p = 0; p < 3; ++p) {
    g.n[p] = P->n[p];
    g.hh[p] = P->hh[p];
  }
  {
    long total = (long)M * 6 * P->glen;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    DEMAG_LAUNCH(P, kFamSetup, st, generators_kernel<<<blocks, 256, 0, st>>>(M, P->glen, g, P->nodes, P->gen64));
    TRY_CUDA(cudaGetLastError());
  }
  if (fft_ok) {
    TRY_CUDA(cudaMalloc(&P->sym, sizeof(float) * (size_t)M * 6 * (P->Lmax / 2 + 1)));
    TRY_CUDA(cudaMemsetAsync(P->sym, 0, sizeof(float) * (size_t)M * 6 * (P->Lmax / 2 + 1), st));
    for (int p = 0; p < 3; ++p) {
      int same = -1;
      for (int q = 0; q < p; ++q)
        if (P->L[q] == P->L[p]) same = q;
      if (same >= 0) {
        P->twid[p] = P->twid[same];
      } else {
        TRY_CUDA(cudaMalloc(&P->twid[p], sizeof(float2) * P->L[p]));
        DEMAG_LAUNCH(P, kFamSetup, st, twiddle_kernel<<<(P->L[p] + 255) / 256, 256, 0, st>>>(P->L[p], P->twid[p]));
        TRY_CUDA(cudaGetLastError());
      }
      dispatch_symbol(P, p, P->M, 2, P->gen64, P->sym, st);
      TRY_CUDA(cudaGetLastError());
    }
    TRY_CUDA(cudaMalloc(&P->sympair, sizeof(float2) * (size_t)M * 6 * (P->Lmax / 2)));
    for (int p = 0; p < 3; ++p) {
      const int N = P->L[p] / 2;
      const long total = (long)M * 2 * N;
      int blocks = (int)((total + 255) / 256);
      if (blocks > 152 * 16) blocks = 152 * 16;
      DEMAG_LAUNCH(P, kFamSetup, st,
                   sympair_kernel<<<blocks, 256, 0, st>>>(M, 2, p, N, P->Lmax / 2 + 1, P->Lmax / 2, P->sym,
                                                          P->sympair));
      TRY_CUDA(cudaGetLastError());
    }
  }
  TRY_CUDA(cudaStreamSynchronize(st));
#undef TRY_CUDA
  *out = P;
  return DEMAG_OK;
}

extern "C" demag_status demag_build_factors_nonuniform(const demag_grid_edges_desc* d, demag_plan** out,
                                                       void* stream) {
  if (!out) return set_error(nullptr, DEMAG_EINVAL, "demag_build_factors_nonuniform: out is NULL");
  *out = nullptr;
  if (!d) return set_error(nullptr, DEMAG_EINVAL, "demag_build_factors_nonuniform: desc is NULL");
  for (int p = 0; p < 3; ++p) {
    if (d->n[p] < 1) return set_error(nullptr, DEMAG_EINVAL, "n[%d] = %d must be >= 1", p, d->n[p]);
    if (d->n[p] > (1 << 20)) return set_error(nullptr, DEMAG_EUNSUPPORTED, "n[%d] too large", p);
    if (!d->edges[p]) return set_error(nullptr, DEMAG_EINVAL, "edges[%d] is NULL", p);
    for (int j = 0; j <= d->n[p]; ++j)
      if (!std::isfinite(d->edges[p][j]) || (j > 0 && !(d->edges[p][j] > d->edges[p][j - 1])))
        return set_error(nullptr, DEMAG_EINVAL, "edges[%d] must be finite and strictly increasing", p);
  }
  if (d->R < 5 || d->R % 2 == 0)
    return set_error(nullptr, DEMAG_EINVAL, "R = %d must be odd and >= 5 (R = 2M+1)", d->R);
  if ((d->R - 1) / 2 > kMaxTerms)
    return set_error(nullptr, DEMAG_EUNSUPPORTED, "R = %d exceeds 2*%d+1", d->R, kMaxTerms);
  if (!(d->c0 > 0.0) || !std::isfinite(d->c0))
    return set_error(nullptr, DEMAG_EINVAL, "c0 must be positive and finite");

  cudaStream_t st = (cudaStream_t)stream;
  demag_plan* P = new (std::nothrow) demag_plan();
  if (!P) return set_error(nullptr, DEMAG_ENOMEM, "host allocation failed");
  snprintf(P->err, sizeof(P->err), "no error");
  P->serial = g_next_serial.fetch_add(1);
  P->nonuniform = true;
  P->R = d->R;
  P->M = (d->R - 1) / 2;
  P->c0 = d->c0;
  P->s = 0.0;
  P->nmax = 0;
  P->Lmax = 0;
  for (int p = 0; p < 3; ++p) {
    const double len = d->edges[p][d->n[p]] - d->edges[p][0];
    P->n[p] = d->n[p];
    P->h[p] = len / d->n[p];  // mean cell width (informational)
    P->s = fmax(P->s, len);
    P->nmax = P->n[p] > P->nmax ? P->n[p] : P->nmax;
  }
  for (int p = 0; p < 3; ++p) {
    P->hh[p] = P->h[p] / P->s;
    int L = next_pow2(2 * P->n[p] - 1);
    P->L[p] = L < 2 ? 2 : L;
    P->Lmax = P->L[p] > P->Lmax ? P->L[p] : P->Lmax;
  }
  P->glen = 2 * P->nmax - 1;
  P->tgroup = 0;
  for (int p = 0; p < 3; ++p) {
    P->toff[p] = P->tgroup;
    P->tgroup += (size_t)P->n[p] * P->n[p];
  }
  const int M = P->M;
  double* ydev = nullptr;
  auto fail = [&](demag_status s) {
    snprintf(g_err, sizeof(g_err), "%s", P->err);
    cudaFree(ydev);
    free_plan_buffers(P);
    delete P;
    return s;
  };
#define TRY_CUDA(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fail(cuda_error(P, e_, #call)); \
  } while (0)
  TRY_CUDA(cudaMalloc(&P->nodes, sizeof(double) * 3 * M));
  TRY_CUDA(cudaMalloc(&P->scale, sizeof(double) * M));
  TRY_CUDA(cudaMalloc(&P->dev_status, sizeof(int)));
  TRY_CUDA(cudaMemsetAsync(P->dev_status, 0, sizeof(int), st));
  DEMAG_LAUNCH(P, kFamSetup, st, nodes_kernel<<<(M + 63) / 64, 64, 0, st>>>(M, P->c0, kCPot * P->s, P->nodes, P->scale));
  TRY_CUDA(cudaGetLastError());
  // edges scaled by the longest domain edge, the three axes concatenated
  std::vector<double> y;
  int yoff[3];
  for (int p = 0; p < 3; ++p) {
    yoff[p] = (int)y.size();
    for (int j = 0; j <= P->n[p]; ++j) y.push_back(d->edges[p][j] / P->s);
  }
  TRY_CUDA(cudaMalloc(&ydev, sizeof(double) * y.size()));
  TRY_CUDA(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, st));
  const size_t total = (size_t)M * 2 * P->tgroup;
  TRY_CUDA(cudaMalloc(&P->fac64, sizeof(double) * total));
  {
    size_t blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 nonuniform_factor_kernel<<<(int)blocks, 256, 0, st>>>(M, P->n[0], P->n[1], P->n[2], P->tgroup,
                                                                      P->toff[1], P->toff[2], yoff[1], yoff[2],
                                                                      P->nodes, ydev, P->fac64));
    TRY_CUDA(cudaGetLastError());
  }
  TRY_CUDA(cudaStreamSynchronize(st));
#undef TRY_CUDA
  cudaFree(ydev);
  *out = P;
  return DEMAG_OK;
}

extern "C" void demag_plan_destroy(demag_plan* plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan_buffers(plan);
  delete plan;
}

extern "C" int demag_num_terms(const demag_plan* plan) { return plan ? plan->M : -1; }

extern "C" const char* demag_last_error(const demag_plan* plan) { return plan ? plan->err : g_err; }

extern "C" size_t demag_generators_size(const demag_plan* plan) {
  return plan ? (size_t)plan->M * 6 * plan->glen : 0;
}

extern "C" size_t demag_symbols_size(const demag_plan* plan) {
  return plan ? (size_t)plan->M * 6 * (plan->Lmax / 2 + 1) : 0;
}

static demag_status copy_out(const demag_plan* plan, void* dst, const void* src, size_t bytes,
                             void* stream, const char* what) {
  demag_plan* P = const_cast<demag_plan*>(plan);
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "%s: plan is NULL", what);
  if (!dst) return set_error(P, DEMAG_EINVAL, "%s: dst is NULL", what);
  if (!src) return set_error(P, DEMAG_EUNSUPPORTED, "%s: not built for this grid", what);
  cudaStream_t st = (cudaStream_t)stream;
  DEMAG_CUDA(P, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, st));
  DEMAG_CUDA(P, cudaStreamSynchronize(st));
  return DEMAG_OK;
}

extern "C" demag_status demag_copy_nodes(const demag_plan* plan, double* dst, void* stream) {
  return copy_out(plan, dst, plan ? plan->nodes : nullptr, plan ? sizeof(double) * 3 * plan->M : 0,
                  stream, "demag_copy_nodes");
}

extern "C" demag_status demag_copy_generators(const demag_plan* plan, double* dst, void* stream) {
  return copy_out(plan, dst, plan ? plan->gen64 : nullptr, sizeof(double) * demag_generators_size(plan),
                  stream, "demag_copy_generators");
}

extern "C" demag_status demag_copy_symbols(const demag_plan* plan, float* dst, void* stream) {
  return copy_out(plan, dst, plan ? plan->sym : nullptr, sizeof(float) * demag_symbols_size(plan),
                  stream, "demag_copy_symbols");
}

extern "C" demag_status demag_sync_status(demag_plan* plan, void* stream) {
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "demag_sync_status: plan is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int h = 0;
  DEMAG_CUDA(plan, cudaMemcpyAsync(&h, plan->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  DEMAG_CUDA(plan, cudaStreamSynchronize(st));
  if (h != 0) {
    DEMAG_CUDA(plan, cudaMemsetAsync(plan->dev_status, 0, sizeof(int), st));
    DEMAG_CUDA(plan, cudaStreamSynchronize(st));
    return set_error(plan, (demag_status)h, "device reported status %d (a bounded wait gave up)", h);
  }
  return tc_sync_status(plan, st);
}

extern "C" unsigned long long demag_launch_count(const demag_plan* plan) { return plan ? plan->launches : 0ULL; }

extern "C" demag_status demag_set_wait_limit(demag_plan* plan, double seconds) {
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "demag_set_wait_limit: plan is NULL");
  if (!(seconds >= 0.0 && seconds <= 60.0))
    return set_error(plan, DEMAG_EINVAL, "demag_set_wait_limit: %g s is outside [0, 60]", seconds);
  plan->wait_ns = (unsigned long long)(seconds * 1e9);
  return DEMAG_OK;
}

extern "C" demag_status demag_set_fused(demag_plan* plan, int enable) {
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "demag_set_fused: plan is NULL");
  plan->fused = enable != 0;
  return DEMAG_OK;
}

extern "C" int demag_forward_schedule(const demag_plan* plan, demag_precision prec) {
  if (!plan || (prec != DEMAG_BF16X3 && prec != DEMAG_TF32X3)) return -1;
  return tc_forward_schedule(plan, prec);
}

extern "C" demag_status demag_autotune(demag_plan* plan, int enable) {
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "demag_autotune: plan is NULL");
  plan->autotune = enable != 0;
  return DEMAG_OK;
}

extern "C" int demag_autotune_count(const demag_plan* plan) { return plan ? (int)plan->tuned.size() : 0; }

extern "C" demag_status demag_autotune_entry(const demag_plan* plan, int i, int* kind, int key[3], int* value,
                                             float* ms, float* ms_default) {
  if (!plan || i < 0 || i >= (int)plan->tuned.size())
    return set_error(nullptr, DEMAG_EINVAL, "demag_autotune_entry: no entry %d", i);
  const demag_plan::Tuned& t = plan->tuned[i];
  if (kind) *kind = t.kind;
  if (key)
    for (int j = 0; j < 3; ++j) key[j] = t.key[j];
  if (value) *value = t.value;
  if (ms) *ms = t.ms;
  if (ms_default) *ms_default = t.ms_default;
  return DEMAG_OK;
}

// "GPU-xxxxxxxx-xxxx-xxxx-xxxx-xxxxxxxxxxxx" of the current device (as nvidia-smi prints it).
static bool current_gpu_uuid(char* out, size_t len) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
  const unsigned char* u = reinterpret_cast<const unsigned char*>(prop.uuid.bytes);
  snprintf(out, len, "GPU-%02x%02x%02x%02x-%02x%02x-%02x%02x-%02x%02x-%02x%02x%02x%02x%02x%02x", u[0], u[1], u[2],
           u[3], u[4], u[5], u[6], u[7], u[8], u[9], u[10], u[11], u[12], u[13], u[14], u[15]);
  return true;
}

static const char* kTuneLine =
    "{\"gpu\":\"%s\",\"n\":[%d,%d,%d],\"R\":%d,\"grid\":\"%s\",\"kind\":%d,\"key\":[%d,%d,%d],"
    "\"value\":%d,\"ms\":%.6g,\"ms_default\":%.6g}\n";

extern "C" demag_status demag_autotune_save(const demag_plan* plan, const char* path) {
  if (!plan || !path) return set_error(nullptr, DEMAG_EINVAL, "demag_autotune_save: NULL argument");
  char gpu[64];
  if (!current_gpu_uuid(gpu, sizeof(gpu)))
    return set_error(const_cast<demag_plan*>(plan), DEMAG_ECUDA, "demag_autotune_save: no device");
  FILE* f = fopen(path, "a");
  if (!f) return set_error(const_cast<demag_plan*>(plan), DEMAG_EINVAL, "demag_autotune_save: cannot open %s", path);
  for (const demag_plan::Tuned& t : plan->tuned)
    fprintf(f, kTuneLine, gpu, plan->n[0], plan->n[1], plan->n[2], plan->R,
            plan->nonuniform ? "nonuniform" : "uniform", t.kind, t.key[0], t.key[1], t.key[2], t.value, t.ms,
            t.ms_default);
  fclose(f);
  return DEMAG_OK;
}

extern "C" demag_status demag_autotune_load(demag_plan* plan, const char* path, int* loaded) {
  if (loaded) *loaded = 0;
  if (!plan || !path) return set_error(nullptr, DEMAG_EINVAL, "demag_autotune_load: NULL argument");
  char gpu[64];
  if (!current_gpu_uuid(gpu, sizeof(gpu))) return set_error(plan, DEMAG_ECUDA, "demag_autotune_load: no device");
  FILE* f = fopen(path, "r");
  if (!f) return DEMAG_OK;  // no cache yet
  char line[512];
  int count = 0;
  while (fgets(line, sizeof(line), f)) {
    char g[64], grid[16];
    int n[3], R, kind, key[3], value;
    float ms = 0.f, msd = 0.f;
    const int got = sscanf(line,
                           "{\"gpu\":\"%63[^\"]\",\"n\":[%d,%d,%d],\"R\":%d,\"grid\":\"%15[^\"]\",\"kind\":%d,"
                           "\"key\":[%d,%d,%d],\"value\":%d,\"ms\":%f,\"ms_default\":%f}",
                           g, &n[0], &n[1], &n[2], &R, grid, &kind, &key[0], &key[1], &key[2], &value, &ms, &msd);
    if (got != 13 || strcmp(g, gpu) != 0 || n[0] != plan->n[0] || n[1] != plan->n[1] || n[2] != plan->n[2] ||
        R != plan->R || strcmp(grid, plan->nonuniform ? "nonuniform" : "uniform") != 0)
      continue;
    demag_plan::Tuned t;
    t.kind = kind;
    for (int j = 0; j < 3; ++j) t.key[j] = key[j];
    t.value = value;
    t.ms = ms;
    t.ms_default = msd;
    bool replaced = false;  // a later line for the same shape wins
    for (demag_plan::Tuned& e : plan->tuned)
      if (e.kind == t.kind && e.key[0] == t.key[0] && e.key[1] == t.key[1] && e.key[2] == t.key[2]) {
        e = t;
        replaced = true;
      }
    if (!replaced) plan->tuned.push_back(t);
    ++count;
  }
  fclose(f);
  if (loaded) *loaded = count;
  return DEMAG_OK;
}

extern "C" demag_status demag_profile(demag_plan* plan, int enable) {
  if (!plan) return set_error(nullptr, DEMAG_EINVAL, "demag_profile: plan is NULL");
  plan->prof_on = enable != 0;
  if (enable) {  // a new record; disabling keeps the record for demag_profile_read
    plan->prof.clear();
    plan->prof_used = 0;
  }
  return DEMAG_OK;
}

extern "C" long long demag_profile_count(const demag_plan* plan) { return plan ? (long long)plan->prof.size() : 0; }

extern "C" demag_status demag_profile_launch(demag_plan* plan, long long i, int* family, double* ms) {
  if (!plan || !family || !ms || i < 0 || i >= (long long)plan->prof.size())
    return set_error(plan, DEMAG_EINVAL, "demag_profile_launch: no record %lld", i);
  auto& r = plan->prof[(size_t)i];
  DEMAG_CUDA(plan, cudaEventSynchronize(r.b));
  float t = 0.f;
  DEMAG_CUDA(plan, cudaEventElapsedTime(&t, r.a, r.b));
  *family = r.family;
  *ms = t;
  return DEMAG_OK;
}

extern "C" demag_status demag_profile_read(demag_plan* plan, int family, double* total_ms, long long* launches) {
  if (!plan || !total_ms || !launches) return set_error(plan, DEMAG_EINVAL, "demag_profile_read: NULL argument");
  double t = 0.0;
  long long c = 0;
  for (auto& r : plan->prof) {
    if (r.family != family) continue;
    DEMAG_CUDA(plan, cudaEventSynchronize(r.b));
    float ms = 0.f;
    DEMAG_CUDA(plan, cudaEventElapsedTime(&ms, r.a, r.b));
    t += ms;
    ++c;
  }
  *total_ms = t;
  *launches = c;
  return DEMAG_OK;
}
