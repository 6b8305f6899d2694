// Internal declarations of libdemag (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/demag.h"

namespace demag {

// M <= 256 (R <= 513): the rule is not uniform in h (Remark after Lemma 2), so
// R grows with n; M = 256 gives tau_max ~ 7.6e4, enough for n = 4096.
constexpr int kMaxTerms = 256;
// the compression of Alg. 2 holds M x M Gram matrices in shared memory
constexpr int kMaxCompressTerms = 64;
constexpr int kMaxFFTLog = 13;      // complex FFT length N = L/2 <= 8192 -> n <= 8192
constexpr double kPi = 3.141592653589793238462643383279502884;
// c = 1/(2 pi^{3/2}): (1/4pi) from Eq. coll times 2/sqrt(pi) from Eq. gauss_trans
constexpr double kCPot = 0.08979356106258328;

// Workspace of the full-format path for one precision.
struct Workspace {
  void* base = nullptr;
  size_t bytes = 0;
};

}  // namespace demag

struct demag_plan {
  int n[3];
  double h[3];
  int R, M;
  double c0;
  double s;         // length scale: longest domain edge
  double hh[3];     // scaled cell sizes h_p / s
  int L[3];         // FFT length per axis (power of 2 >= 2 n_p - 1, >= 2)
  int nmax, Lmax;
  int glen;         // generator row length 2*nmax - 1
  unsigned long long serial = 0;  // unique per plan in the process (cache keys)

  // setup data (device)
  double* nodes = nullptr;   // [3][M]: t, tau, omega
  double* gen64 = nullptr;   // [M][2][3][glen]
  float* sym = nullptr;      // [M][2][3][Lmax/2 + 1] symbols / L_p
  float2* twid[3] = {nullptr, nullptr, nullptr};  // per axis: exp(-2 pi i m / L_p), m < L_p
  float2* sympair = nullptr; // [M][2][3][Lmax/2]: (symbol[f], symbol[L_p/2 - f]) for f < L_p/2
  double* scale = nullptr;   // [M]: c * s * omega_k
  double* gend = nullptr;    // [M][2][3][glen]: derivative generators dE/s, dF/s (lazily, analytic stray field)

  // dense factor matrices of the full path, per precision (device, lazily built)
  // layout [M][2][3] blocks of n_p x n_p (row-major T[i][j] = gen[i-j]),
  // axis-3 blocks carry the scale c*s*omega_k.
  float* T32 = nullptr;
  double* T64 = nullptr;
  // non-uniform tensor grid (demag_build_factors_nonuniform): the factors are
  // dense, not Toeplitz.  fac64 holds them in FP64 in the T64 layout without
  // the scale; gen64, sym and the twiddles stay unset (no FFT forms).
  bool nonuniform = false;
  double* fac64 = nullptr;   // [M][2][tgroup]
  float* T32t = nullptr;     // transposed tables for the adjoint (CUDA cores)
  double* T64t = nullptr;
  float* T32d = nullptr;     // the same layout from the derivative generators (analytic stray field)
  double* T64d = nullptr;
  size_t toff[3];            // element offset of axis p inside one (k, type) group
  size_t tgroup;             // elements per (k, type) group = sum_p n_p^2

  demag::Workspace ws[4];    // per demag_precision
  int* dev_status = nullptr; // device status word (DEMAG_ETIMEOUT etc.)
  // tensor-core state (opaque, owned by full_tc.cu)
  void* tc = nullptr;
  // 3D FFT convolution state (opaque, owned by fft3d.cu): dense Fourier kernel and spectra
  void* f3 = nullptr;
  // compressed (Tucker) kernels of Alg. 2 (opaque, owned by compress.cu)
  void* cmp = nullptr;
  // energy / gradient scratch: phi, D^T m (1 field each) and P^T D^T m (3 fields)
  float* ews = nullptr;
  // per-fibre full format: two work volumes of 3M fields each
  float* fib_ws = nullptr;

  // limit of the bounded device-side waits of the tensor-core kernels (ns)
  unsigned long long wait_ns = 2000000000ull;
  // full-format forward application on tensor cores: 1 fuses the mode-1 and
  // mode-2 products where the grid allows it, 0 runs the three-stage chain,
  // -1 (default) the tuned choice (fused when nothing was tuned)
  int fused = -1;

  // autotuning: when on, launch shapes not yet tuned are timed on first use
  bool autotune = false;
  struct Tuned {
    int kind;      // 0 FFT nodes per block; tensor cores (BF16x3 / TF32x3): 1 / 2 N tile,
                   // 3 / 4 operand stages, 5 / 6 tile order, 7 / 8 store boxes;
                   // 9 forward schedule (BF16x3: 1 fused, 0 chain)
    int key[3];    // FFT: log2 N, column blocks, M; tensor core: stage program, default value, 0
    int value;     // chosen setting
    float ms;      // its time per launch
    float ms_default = 0.f;  // the default setting's time per launch (0: not timed, a loaded entry)
  };
  std::vector<Tuned> tuned;

  // diagnostics: kernels launched, and optional CUDA-event timing per family
  unsigned long long launches = 0;
  bool prof_on = false;
  struct ProfRec { int family; cudaEvent_t a, b; };
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> prof_pool;
  size_t prof_used = 0;

  char err[512];
};

namespace demag {

// kernel families for demag_profile_read
enum Family { kFamGemmSimt = 0, kFamGemmTc = 1, kFamFFT = 2, kFamSplit = 3, kFamSetup = 4, kFamEnergy = 5, kFamMisc = 6,
             kFamFFT3D = 7 };

void prof_begin(demag_plan* P, int family, cudaStream_t st);
void prof_end(demag_plan* P, cudaStream_t st);

// Bracket one kernel launch: counts it and, when profiling is on, records
// CUDA events around it on the launching stream.
#define DEMAG_LAUNCH(P, family, st, ...)     \
  do {                                       \
    demag::prof_begin((P), (family), (st));  \
    __VA_ARGS__;                             \
    (P)->launches++;                         \
    demag::prof_end((P), (st));              \
  } while (0)

// error helpers ---------------------------------------------------------------
demag_status set_error(demag_plan* plan, demag_status st, const char* fmt, ...);
demag_status cuda_error(demag_plan* plan, cudaError_t e, const char* where);

#define DEMAG_CUDA(plan, call)                                  \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return demag::cuda_error(plan, e_, #call); \
  } while (0)

#define DEMAG_LAUNCHED(plan, what)                              \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return demag::cuda_error(plan, e_, what); \
  } while (0)

inline size_t field_size(const demag_plan* p) { return (size_t)p->n[0] * p->n[1] * p->n[2]; }

// full format (full_simt.cu / full_tc.cu) ---------------------------------------
demag_status ensure_dense_factors(demag_plan* plan, demag_precision prec, cudaStream_t st);
demag_status ensure_field_generators(demag_plan* plan, cudaStream_t st);
demag_status simt_field(demag_plan* plan, const float* m, float* hd, demag_precision prec, cudaStream_t st);
demag_status tc_field(demag_plan* plan, const float* m, float* hd, demag_precision prec, cudaStream_t st);
demag_status ensure_workspace(demag_plan* plan, demag_precision prec);
size_t workspace_bytes(const demag_plan* plan, demag_precision prec);
demag_status full_forward(demag_plan* plan, const float* m, float* phi, demag_precision prec,
                          cudaStream_t st);
demag_status full_adjoint(demag_plan* plan, const float* y, float* g, demag_precision prec,
                          cudaStream_t st);

// tensor cores (full_tc.cu)
demag_status tc_prepare(demag_plan* plan, demag_precision prec, cudaStream_t st);
demag_status tc_forward(demag_plan* plan, const float* m, float* phi, demag_precision prec,
                        cudaStream_t st);
demag_status tc_adjoint(demag_plan* plan, const float* y, float* g, demag_precision prec,
                        cudaStream_t st);
struct TcBatch;
demag_status tc_batch_create(demag_plan* const* plans, int count, demag_precision prec, TcBatch** out);
demag_status tc_batch_run(const TcBatch* batch, const float* const* m, float* const* phi, cudaStream_t st);
void tc_batch_destroy(TcBatch* batch);
demag_status tc_forward_batched(demag_plan* const* plans, const float* const* m, float* const* phi, int count,
                                demag_precision prec, cudaStream_t st);
size_t tc_workspace_bytes(const demag_plan* plan, demag_precision prec);
demag_status tc_sync_status(demag_plan* plan, cudaStream_t st);
bool tc_ready(const demag_plan* plan, demag_precision prec);
// forward schedule of a prepared plan: 1 fused, 0 three-stage chain, -1 no tensor-core state
int tc_forward_schedule(const demag_plan* plan, demag_precision prec);
void tc_destroy(demag_plan* plan);

// compressed kernels (compress.cu)
struct CompressedView {
  int rho[3];
  const float2* cpair;  // symbol pairs [rhomax][3 q][3 p][Lmax/2]
  const float* core;    // [3 q][rho3][rho2][rho1]
};
bool compressed_view(const demag_plan* plan, CompressedView* v);
void compress_destroy(demag_plan* plan);
demag_status launch_core_kron(demag_plan* plan, int batch, const int r[3], const float* G, float* out,
                              cudaStream_t st);

// 3D FFT convolution (fft3d.cu)
demag_status fft3d_forward(demag_plan* plan, const float* m, float* phi, cudaStream_t st);
void fft3d_destroy(demag_plan* plan);

// setup kernels (plan.cu)
struct GridInfo {
  int n[3];
  double hh[3];
};
__global__ void nodes_kernel(int M, double c0, double cscale, double* nodes, double* scale);
__global__ void generators_kernel(int M, int glen, GridInfo g, const double* nodes, double* gen);
demag_status require_uniform(demag_plan* plan, const char* what);
void dispatch_symbol(demag_plan* P, int axis, int M, int nsets, const double* gen, float* sym, cudaStream_t st);
__global__ void sympair_kernel(int M, int nsets, int axis, int N, int symstride, int pairstride, const float* sym,
                               float2* pair);
__global__ void nonuniform_factor_kernel(int M, int n0, int n1, int n2, size_t tgroup, size_t off1, size_t off2,
                                         int yoff1, int yoff2, const double* nodes, const double* y, double* fac);

// energy (energy.cu)
demag_status fd_gradient(demag_plan* plan, const float* phi, float* out, float scale,
                         cudaStream_t st);
void energy_destroy(demag_plan* plan);

}  // namespace demag
