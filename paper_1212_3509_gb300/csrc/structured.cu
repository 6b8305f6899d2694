// Structured formats: batched 1D Toeplitz matvecs through circulant FFTs.
//
// Eq. kron_eval_cp / Eq. kron_eval_tuck (Sec. 3.4) and App. C Eq. tt_3d_2:
// applying the Kronecker operator to a CP / Tucker / TT tensor maps every
// factor column v (mode p, component q) to T_{k,q,p} v for each node k.
// Sec. 4.2 (Eq. conv_op, conv_pot, fft_pot) and Lemmas 4-5: with midpoint
// collocation on a uniform grid the factors are Toeplitz, so each matvec is a
// circular convolution of the zero-padded column with the length-L embedding
// of the generator: y = IFFT(FFT(v, L) * symbol)[0:n].  FP32 throughout; the
// symbols were computed in FP64 at setup and carry the 1/L of the inverse.
//
// The real inverse transform of length L = 2N runs as a complex one of
// length N on Z[f] = Y_f (1 + i conj(w_f)) + conj(Y_{N-f}) (1 - i conj(w_f)),
// w_f = exp(-2 pi i f / L), Y = symbol * X.  With the per-column constants
// P[f] = X_f (1 + i conj(w_f)) and Q[f] = conj(X_{N-f}) (1 - i conj(w_f)) this is
//   E (real symbol s):        Z[f] = s_f P[f] + s_{N-f} Q[f]
//   F (imaginary symbol i s): Z[f] = i (s_f P[f] - s_{N-f} Q[f]),
// four multiply-adds per bin.
//
// A group of TG threads owns one column.  It computes P and Q once (shared
// memory) and then, for each node of its node range:
//   pass 1  (registers)  Z for the bins of this thread's first radix pass,
//                        the first radix-R DFT, written to shared memory;
//   middle  (shared)     radix-16 Stockham passes in place (one buffer padded
//                        by one element per 16 so strided writes do not
//                        collide in banks);
//   last    (registers)  final radix-16 pass; only the outputs of the first
//                        half of the complex signal (the n real samples we
//                        keep) are computed and stored to HBM.
// Twiddles: one value per item from a two-level shared table
// (W_L^m = T1[m >> 7] * T0[m & 127]) and its powers by a product tree.
#include <climits>
#include <type_traits>

#include "internal.h"
#include "fft.cuh"

namespace demag {

// One axis of a launch: its columns, input and output layout.
struct ToepAxis {
  int n;           // column length n_p
  int axis;        // p
  int rcols;       // columns per (batch item, component)
  int ncols;       // batch * 3 * rcols
  const float* in; // column (b, q, l) at in + b*in_bstride + q*in_qstride + l*n
  long in_bstride, in_qstride;
  float* out;      // node k: out + b*out_bstride + ((k*3 + q)*rcols + l)*n
  long out_bstride;
  int kmax;        // nodes (generators) of this axis: k < kmax
  const float2* twid;     // exp(-2 pi i m / L), m < L
};

// Every axis whose FFT length is the same goes into one launch: blocks
// [bx0[s], bx0[s+1]) of grid.x serve axis slot s, grid.y covers the nodes.
struct ToepLaunch {
  ToepAxis ax[3];
  int naxes;
  int bx0[4];
  int M;           // number of nodes (the largest kmax)
  int kgroup;      // nodes per block
  int pairstride;  // Lmax/2
  int nsets;       // symbol sets per node: 2 (types E, F) or 3 (components of a compressed kernel)
  int diag;        // 1: column (b, q, l) applies node b only and writes it as node 0 of its item
  const float2* sympair;  // [M][nsets][3][pairstride]: (s_f, s_{N-f}); set = type, or q when nsets = 3
};

template <int LOGN> struct ToepCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr int L = 2 * N;
  // one thread per item of a radix-16 pass, at least 16.  With TG >= 32 the node loop is
  // specialised on the factor type of the column; a group narrower than a warp shares its warp
  // with columns of the other type, so there the type is a runtime value and every thread runs
  // the same code through the block barriers
  static constexpr int TG = (N / 16) < 16 ? 16 : ((N / 16) > 256 ? 256 : (N / 16));
  static constexpr int G = 256 / TG;
  static constexpr int NP = N + N / 16;            // padded buffer length
  static constexpr int T0 = L < 128 ? L : 128;     // fine twiddle table
  static constexpr int T1 = L / T0;                // coarse twiddle table
  static constexpr int R1 = (LOGN % 4) ? (1 << (LOGN % 4)) : (LOGN >= 4 ? 16 : 1);
  static constexpr int NPASS = LOGN / 4 + ((LOGN % 4) ? 1 : 0);
  // per group: P and Q interleaved (N float4) and one padded work buffer (NP float2);
  // layout [G][N] float4 | T0 | T1 | [G][NP] float2
  static constexpr size_t smem = (size_t)G * N * sizeof(float4) + ((size_t)T0 + T1 + (size_t)G * NP) * sizeof(float2);
  static constexpr int minblocks = smem * 2 <= 220 * 1024 ? 2 : 1;
};

struct TwSmem {
  const float2* t0;
  const float2* t1;
  // W_L^m
  __device__ __forceinline__ float2 L(int m) const { return cmul(t1[m >> 7], t0[m & 127]); }
};

// forward-FFT twiddle W_N^m = W_L^(2m) for the generic in-place routine
struct TwN {
  TwSmem s;
  __device__ __forceinline__ float2 operator()(int m) const { return s.L(2 * m); }
};

// The first 8 outputs of an inverse 16-point DFT (the kept half of the last
// pass): two 8-point DFTs of the even and odd inputs and the "+" half of the
// final butterflies.
template <int K>
__device__ __forceinline__ void combine_half16(float2 (&v)[16], float2 (&e)[8], float2 (&o)[8]) {
  if constexpr (K < 8) {
    const float2 t = rot<16, K, true>(o[K]);
    if constexpr (K == 4) {  // +i: folded into scalar adds
      v[K].x = e[K].x + t.x;
      v[K].y = e[K].y + t.y;
    } else {
      v[K] = cadd(e[K], t);
    }
    combine_half16<K + 1>(v, e, o);
  }
}

__device__ __forceinline__ void idft16_first_half(float2 (&v)[16]) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft_reg<8, true>(e);
  dft_reg<8, true>(o);
  combine_half16<0>(v, e, o);
}

// In-place middle pass of radix R on the padded buffer (inverse direction):
// every item is read into registers, the block synchronises, then writes.
template <int R, int N, int TG>
__device__ __forceinline__ void mid_pass(float2* buf, int Ns, int lt, const TwSmem& tw) {
  constexpr int items = N / R;
  constexpr int ipt = (items + TG - 1) / TG;
  float2 v[ipt][R];
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
      float2 w = tw.L(2 * k * (N / (Ns * R)));
      w.y = -w.y;
      float2 pw[R];
      powers<R>(w, pw);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float2 x = (items % 16 == 0) ? buf[pad16(j) + r * PadStride<items>::value] : buf[pad16(j + r * items)];
        v[it][r] = r > 0 ? cmul(x, pw[r]) : x;
      }
      dft_reg<R, true>(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * R + k;
      if (Ns % 16 == 0) {
        const int b0 = pad16(base), step = Ns + (Ns >> 4);
#pragma unroll
        for (int r = 0; r < R; ++r) buf[b0 + r * step] = v[it][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) buf[pad16(base + r * Ns)] = v[it][r];
      }
    }
  }
  __syncthreads();
}

template <int LOGN>
__global__ void __launch_bounds__(256, ToepCfg<LOGN>::minblocks)
    toeplitz_fft_kernel(const __grid_constant__ ToepLaunch a) {
  using Cfg = ToepCfg<LOGN>;
  constexpr int N = Cfg::N, TG = Cfg::TG, R1 = Cfg::R1, NPASS = Cfg::NPASS;
  extern __shared__ float4 smem_c[];
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float4* PQ = smem_c + (size_t)g * N;  // (P_f, Q_f) of this group's column
  float2* t0 = reinterpret_cast<float2*>(smem_c + (size_t)Cfg::G * N);
  float2* t1 = t0 + Cfg::T0;
  float2* buf = t1 + Cfg::T1 + (size_t)g * Cfg::NP;
  int slot = 0;
  while (slot + 1 < a.naxes && (int)blockIdx.x >= a.bx0[slot + 1]) ++slot;
  const ToepAxis& A = a.ax[slot];
  for (int i = threadIdx.x; i < Cfg::T0; i += blockDim.x) t0[i] = __ldg(A.twid + i);
  for (int i = threadIdx.x; i < Cfg::T1; i += blockDim.x) t1[i] = __ldg(A.twid + i * Cfg::T0);
  const TwSmem tw{t0, t1};

  const int c = ((int)blockIdx.x - a.bx0[slot]) * Cfg::G + g;
  const bool active = c < A.ncols;
  const int l = active ? c % A.rcols : 0;
  const int bq = active ? c / A.rcols : 0;
  const int q = bq % 3, b = bq / 3;
  const int n = A.n;
  const int rcols = A.rcols;
  const float* in = A.in + b * A.in_bstride + q * A.in_qstride + (long)l * n;

  // 1. zero-padded column as N complex samples, forward FFT (once per column)
  for (int j = lt; j < N; j += TG) {
    float x0 = 0.f, x1 = 0.f;
    if (active) {
      if (2 * j < n) x0 = __ldg(in + 2 * j);
      if (2 * j + 1 < n) x1 = __ldg(in + 2 * j + 1);
    }
    buf[j] = make_float2(x0, x1);
  }
  __syncthreads();
  fft_inplace<LOGN, TG, false>(buf, lt, TwN{tw});

  // 2. split step to the real spectrum X and the per-column constants P, Q
  for (int f = lt; f < N; f += TG) {
    const int fc = (N - f) & (N - 1);
    const float2 A = buf[f], B = buf[fc];
    const float2 w = tw.L(f);                  // w_f
    const float2 wc = make_float2(-w.x, w.y);  // w_{N-f} = -conj(w_f)
    // X_f = (A + conj B)/2 - i/2 w_f (A - conj B); X_{N-f} with A, B swapped
    float ex = 0.5f * (A.x + B.x), ey = 0.5f * (A.y - B.y);
    float dx = 0.5f * (A.x - B.x), dy = 0.5f * (A.y + B.y);
    float wx = w.x * dx - w.y * dy, wy = w.x * dy + w.y * dx;
    const float2 Xf = make_float2(ex + wy, ey - wx);
    ex = 0.5f * (B.x + A.x);
    ey = 0.5f * (B.y - A.y);
    dx = 0.5f * (B.x - A.x);
    dy = 0.5f * (B.y + A.y);
    wx = wc.x * dx - wc.y * dy;
    wy = wc.x * dy + wc.y * dx;
    const float2 Xc = make_float2(ex + wy, ey - wx);
    // 1 + i conj(w) and 1 - i conj(w)
    const float2 up = make_float2(1.f + w.y, w.x), um = make_float2(1.f - w.y, -w.x);
    const float2 Pf = cmul(Xf, up), Qf = cmul(make_float2(Xc.x, -Xc.y), um);
    PQ[f] = make_float4(Pf.x, Pf.y, Qf.x, Qf.y);
  }
  __syncthreads();

  const int axis = A.axis;
  const int type = (axis == q) ? 1 : 0;  // F on the axis of the component
  const int k0 = a.diag ? b : blockIdx.y * a.kgroup;
  const int k1 = a.diag ? b + 1 : min(min(a.M, A.kmax), k0 + a.kgroup);
  const int kofs = a.diag ? k0 : 0;  // output node index = k - kofs
  float* outbase = A.out + b * A.out_bstride + (long)l * n;
  // paired stores need an even length and an 8-byte aligned column start
  // (every (k, q) offset is a multiple of n, so one check per column)
  const bool vec = ((n & 1) == 0) && ((reinterpret_cast<uintptr_t>(outbase) & 7) == 0);
  // the last pass keeps outputs i < N/2 (as pairs 2i, 2i + 1): all exist when n >= N
  const bool full_vec = vec && n >= N;
  // The last pass's twiddles depend only on the thread's item: with one item
  // per thread they are computed once here and reused for every node.
  constexpr int items_last = N / 16;
  constexpr bool keep_tw = NPASS > 1 && items_last == TG;
  float2 pw_last[keep_tw ? 16 : 1];
  if constexpr (keep_tw) {
    float2 w = tw.L(2 * lt);  // W_N^j with j = lt, inverse: conjugate
    w.y = -w.y;
    powers<16>(w, pw_last);
  }
  // the node loop, specialised on the factor type (E or F), which is fixed per column
  auto node_loop = [&](auto type_tag) {
    constexpr int TYPE = decltype(type_tag)::value;  // 0 E, 1 F, -1 taken from the column at run time
    const int ftype = TYPE < 0 ? type : TYPE;
    for (int k = k0; k < k1; ++k) {
      const float2* sp = a.sympair + ((long)(k * a.nsets + (a.nsets == 3 ? q : ftype)) * 3 + axis) * a.pairstride;
      // 3. first pass in registers on the bins j + r N/R1 of item j
      constexpr int items1 = N / R1;
      constexpr int ipt1 = (items1 + TG - 1) / TG;
  #pragma unroll
      for (int it = 0; it < ipt1; ++it) {
        const int j = lt + it * TG;
        if (items1 % TG == 0 || j < items1) {
          float2 v[R1];
  #pragma unroll
          for (int r = 0; r < R1; ++r) {
            const int f = j + r * items1;
            const float2 s2 = __ldg(sp + f);
            const float4 pq = PQ[f];  // (P, Q)
            // E: s_f P + s_c Q ;  F: i (s_f P - s_c Q)
            const float sc = ftype ? -s2.y : s2.y;
            const float zx = fmaf(s2.x, pq.x, sc * pq.z);
            const float zy = fmaf(s2.x, pq.y, sc * pq.w);
            v[r] = ftype ? make_float2(-zy, zx) : make_float2(zx, zy);
          }
          dft_reg<R1, true>(v);
          if constexpr (NPASS <= 1) {
            // single pass: outputs j + r*items1, keep the first half
  #pragma unroll
            for (int r = 0; r < R1; ++r) {
              const int i = j + r * items1;
              if (active && 2 * i < n) {
                float* o = outbase + (long)((k - kofs) * 3 + q) * rcols * n;
                o[2 * i] = v[r].x;
                if (2 * i + 1 < n) o[2 * i + 1] = v[r].y;
              }
            }
          } else {
  #pragma unroll
            for (int r = 0; r < R1; ++r) buf[pad16(j * R1 + r)] = v[r];
          }
        }
      }
      if constexpr (NPASS > 1) {
        __syncthreads();
        // 4. middle radix-16 passes in place
        int Ns = R1;
  #pragma unroll
        for (int ps = 1; ps < NPASS - 1; ++ps) {
          mid_pass<16, N, TG>(buf, Ns, lt, tw);
          Ns *= 16;
        }
        // 5. last radix-16 pass (Ns = N/16): outputs j + r N/16, keep r < 8
        constexpr int items = N / 16;
        constexpr int ipt = (items + TG - 1) / TG;
  #pragma unroll
        for (int it = 0; it < ipt; ++it) {
          const int j = lt + it * TG;
          if (items % TG == 0 || j < items) {
            float2 v[16];
            float2 pw[16];
            if constexpr (keep_tw) {
  #pragma unroll
              for (int r = 0; r < 16; ++r) pw[r] = pw_last[r];
            } else {
              float2 w = tw.L(2 * j);  // W_N^j (Ns = N/16, so k = j), inverse: conjugate
              w.y = -w.y;
              powers<16>(w, pw);
            }
  #pragma unroll
            for (int r = 0; r < 16; ++r) {
              const float2 x =
                  (items % 16 == 0) ? buf[pad16(j) + r * PadStride<items>::value] : buf[pad16(j + r * items)];
              v[r] = r > 0 ? cmul(x, pw[r]) : x;
            }
            idft16_first_half(v);
            if (active && full_vec) {
              // every kept output exists: 8-byte stores, no bounds tests
              float2* o = reinterpret_cast<float2*>(outbase + (long)((k - kofs) * 3 + q) * rcols * n);
  #pragma unroll
              for (int r = 0; r < 8; ++r) o[j + r * items] = v[r];
            } else if (active) {
              float* o = outbase + (long)((k - kofs) * 3 + q) * rcols * n;
  #pragma unroll
              for (int r = 0; r < 8; ++r) {
                const int i = j + r * items;
                if (2 * i + 1 < n) {
                  if (vec)
                    reinterpret_cast<float2*>(o)[i] = v[r];
                  else {
                    o[2 * i] = v[r].x;
                    o[2 * i + 1] = v[r].y;
                  }
                } else if (2 * i < n) {
                  o[2 * i] = v[r].x;
                }
              }
            }
          }
        }
      }
      __syncthreads();
    }
  };
  if constexpr (TG < 32)
    node_loop(std::integral_constant<int, -1>{});
  else if (type)
    node_loop(std::integral_constant<int, 1>{});
  else
    node_loop(std::integral_constant<int, 0>{});
}

// weights: out_w[b][k][q][l] = c s omega_k * lambda[b][q][l] (lambda NULL -> 1)
__global__ void weights_kernel(int M, int batch, int rq, const double* scale, const float* lambda,
                               float* out_w) {
  long total = (long)batch * M * 3 * rq;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    int l = (int)(i % rq);
    long t = i / rq;
    int q = (int)(t % 3);
    t /= 3;
    int k = (int)(t % M);
    int b = (int)(t / M);
    double lam = lambda ? (double)lambda[((long)b * 3 + q) * rq + l] : 1.0;
    out_w[i] = (float)(scale[k] * lam);
  }
}

template <int LOGN>
static cudaError_t launch_toep(demag_plan* P, const ToepLaunch& a, int gx, cudaStream_t st) {
  using Cfg = ToepCfg<LOGN>;
  if (Cfg::smem > 48 * 1024) {
    // once per device (so that later launches, e.g. under stream capture,
    // make no attribute calls)
    static unsigned long long done = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(done & bit)) {
      cudaError_t e = cudaFuncSetAttribute(toeplitz_fft_kernel<LOGN>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem);
      if (e != cudaSuccess) return e;
      done |= bit;
    }
  }
  int gy = (a.M + a.kgroup - 1) / a.kgroup;
  DEMAG_LAUNCH(P, kFamFFT, st, toeplitz_fft_kernel<LOGN><<<dim3(gx, gy), 256, Cfg::smem, st>>>(a));
  return cudaGetLastError();
}

static int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

static int groups_per_block(int logn) {
  int N = 1 << logn;
  int TG = N / 16 < 16 ? 16 : (N / 16 > 256 ? 256 : N / 16);
  return 256 / TG;
}

static cudaError_t launch_logn(demag_plan* P, int logn, const ToepLaunch& a, int gx, cudaStream_t st) {
  switch (logn) {
    case 0: return launch_toep<0>(P, a, gx, st);
    case 1: return launch_toep<1>(P, a, gx, st);
    case 2: return launch_toep<2>(P, a, gx, st);
    case 3: return launch_toep<3>(P, a, gx, st);
    case 4: return launch_toep<4>(P, a, gx, st);
    case 5: return launch_toep<5>(P, a, gx, st);
    case 6: return launch_toep<6>(P, a, gx, st);
    case 7: return launch_toep<7>(P, a, gx, st);
    case 8: return launch_toep<8>(P, a, gx, st);
    case 9: return launch_toep<9>(P, a, gx, st);
    case 10: return launch_toep<10>(P, a, gx, st);
    case 11: return launch_toep<11>(P, a, gx, st);
    case 12: return launch_toep<12>(P, a, gx, st);
    case 13: return launch_toep<13>(P, a, gx, st);
    default: return cudaErrorInvalidValue;
  }
}

// Nodes per block.  Each block transforms its columns once and reuses the
// spectra for kgroup nodes, so large groups save forward FFTs, while small
// groups give more blocks.  Default: the largest group that still yields
// eight blocks per SM; with autotuning on, the candidates M, M/2, M/4, ..., 1
// are timed once per (FFT length, column blocks, M) and the fastest is kept.
static cudaError_t pick_kgroup(demag_plan* P, int logn, ToepLaunch& a, int gx, cudaStream_t st) {
  const int M = a.M;
  for (const demag_plan::Tuned& t : P->tuned)
    if (t.kind == 0 && t.key[0] == logn && t.key[1] == gx && t.key[2] == M) {
      a.kgroup = t.value;
      return cudaSuccess;
    }
  int kg = M;
  while (kg > 1 && (long)gx * ((M + kg - 1) / kg) < 1216) kg = (kg + 1) / 2;
  a.kgroup = kg;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cap);
  if (!P->autotune || cap != cudaStreamCaptureStatusNone) return cudaSuccess;
  std::vector<int> cands;
  for (int c = M;; c = (c + 1) / 2) {
    if (cands.empty() || cands.back() != c) cands.push_back(c);
    if (c == 1) break;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f, at_def = 0.f;
  int best_kg = kg;
  cudaError_t err = cudaSuccess;
  for (int c : cands) {
    a.kgroup = c;
    err = launch_logn(P, logn, a, gx, st);  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && err == cudaSuccess; ++r) err = launch_logn(P, logn, a, gx, st);
    cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (c == kg) at_def = ms;
    if (ms < best) {
      best = ms;
      best_kg = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return err;
  a.kgroup = best_kg;
  demag_plan::Tuned t;
  t.kind = 0;
  t.key[0] = logn;
  t.key[1] = gx;
  t.key[2] = M;
  t.value = best_kg;
  t.ms = best / 3.f;
  t.ms_default = at_def / 3.f;
  P->tuned.push_back(t);
  return cudaSuccess;
}

// Toeplitz matvecs of the given axes: axes that share an FFT length run in
// one launch (normally all three), each as its own range of blocks.
static demag_status run_axes(demag_plan* P, ToepAxis* axes, int count, const char* what, cudaStream_t st,
                             const float2* sympair = nullptr, int nsets = 2, int diag = 0) {
  bool done[3] = {false, false, false};
  for (int i = 0; i < count; ++i) {
    if (done[i]) continue;
    const int logn = ilog2i(P->L[axes[i].axis] / 2);
    const int G = groups_per_block(logn);
    ToepLaunch a{};
    a.M = 0;
    a.pairstride = P->Lmax / 2;
    a.sympair = sympair ? sympair : P->sympair;
    a.nsets = nsets;
    int gx = 0;
    for (int j = i; j < count; ++j) {
      if (done[j] || ilog2i(P->L[axes[j].axis] / 2) != logn) continue;
      ToepAxis x = axes[j];
      x.n = P->n[x.axis];
      x.twid = P->twid[x.axis];
      if (x.kmax <= 0) x.kmax = P->M;
      a.M = x.kmax > a.M ? x.kmax : a.M;
      a.ax[a.naxes] = x;
      a.bx0[a.naxes] = gx;
      gx += (x.ncols + G - 1) / G;
      ++a.naxes;
      done[j] = true;
    }
    a.bx0[a.naxes] = gx;
    a.diag = diag;
    cudaError_t e = cudaSuccess;
    if (diag)
      a.kgroup = a.M;  // one node per column: grid.y = 1
    else
      e = pick_kgroup(P, logn, a, gx, st);
    if (e == cudaSuccess) e = launch_logn(P, logn, a, gx, st);
    if (e != cudaSuccess) return cuda_error(P, e, what);
  }
  return DEMAG_OK;
}

static demag_status check_fft_plan(demag_plan* P, const char* what) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "%s: plan is NULL", what);
  demag_status u = require_uniform(P, what);  // Toeplitz factors only
  if (u != DEMAG_OK) return u;
  if (!P->sym || !P->sympair)
    return set_error(P, DEMAG_EUNSUPPORTED, "%s: n_p up to %d supported by the FFT path", what,
                     1 << kMaxFFTLog);
  return DEMAG_OK;
}

static demag_status launch_weights(demag_plan* P, int batch, int rq, const float* lambda, float* out_w,
                                   cudaStream_t st) {
  long total = (long)batch * P->M * 3 * rq;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  DEMAG_LAUNCH(P, kFamMisc, st, weights_kernel<<<blocks, 256, 0, st>>>(P->M, batch, rq, P->scale, lambda, out_w));
  DEMAG_LAUNCHED(P, "weights_kernel");
  return DEMAG_OK;
}

// ---------------------------------------------------------------- full format by per-fibre Toeplitz FFTs
//
// phi = c s sum_k omega_k sum_q T_{k,q,3} x_3 T_{k,q,2} x_2 T_{k,q,1} x_1 m^(q) (Eq. kron_operator) with
// every mode product done as 1D Toeplitz matvecs of the fibres through the circulant FFT kernel
// (Sec. 4.2): axis 1 for all nodes at once (one forward FFT per fibre), then axes 2 and 3 per
// (node, component) volume (diagonal mode), with batched transposes between so that every FFT
// reads contiguous fibres, and a weighted sum over (k, q) that transposes back.

// out[b][c][r] = in[b][r][c]: 32 x 32 tiles through shared memory, grid-stride over all tiles
__global__ void __launch_bounds__(256) transpose_batched_kernel(long B, int R, int C, const float* in, float* out) {
  __shared__ float tile[32][33];
  const int tr = (R + 31) / 32, tc = (C + 31) / 32;
  const long total = B * tr * tc;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (long t = blockIdx.x; t < total; t += gridDim.x) {
    const long b = t / ((long)tr * tc);
    const int rem = (int)(t - b * tr * tc);
    const int r0 = (rem / tc) * 32, c0 = (rem % tc) * 32;
    const float* src = in + b * (long)R * C;
    float* dst = out + b * (long)R * C;
    for (int i = ty; i < 32; i += 8) {
      const int r = r0 + i, c = c0 + tx;
      tile[i][tx] = (r < R && c < C) ? src[(long)r * C + c] : 0.f;
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int c = c0 + i, r = r0 + tx;
      if (r < R && c < C) dst[(long)c * R + r] = tile[tx][i];
    }
    __syncthreads();
  }
}

// phi[i3][i2][i1] = sum_{k, q} scale[k] Y[k][q][i1][i2][i3]: per i2 a 32 x 32 (i1, i3) tile,
// read along i3 and written along i1
__global__ void __launch_bounds__(256) fibre_sum_kernel(int M, int n1, int n2, int n3, const double* scale,
                                                        const float* Y, float* phi) {
  __shared__ float tile[32][33];
  const int t1 = (n1 + 31) / 32, t3 = (n3 + 31) / 32;
  const long total = (long)n2 * t1 * t3;
  const long N = (long)n1 * n2 * n3;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (long t = blockIdx.x; t < total; t += gridDim.x) {
    const int i2 = (int)(t / ((long)t1 * t3));
    const int rem = (int)(t - (long)i2 * t1 * t3);
    const int a0 = (rem / t3) * 32, c0 = (rem % t3) * 32;  // i1 and i3 tile origins
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k = 0; k < M; ++k) {
      const float w = (float)scale[k];
      for (int q = 0; q < 3; ++q) {
        const float* src = Y + ((long)k * 3 + q) * N;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i1 = a0 + ty + 8 * u, i3 = c0 + tx;
          if (i1 < n1 && i3 < n3) acc[u] = fmaf(w, src[((long)i1 * n2 + i2) * n3 + i3], acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) tile[ty + 8 * u][tx] = acc[u];
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int i3 = c0 + i, i1 = a0 + tx;
      if (i1 < n1 && i3 < n3) phi[((long)i3 * n2 + i2) * n1 + i1] = tile[tx][i];
    }
    __syncthreads();
  }
}

static int grid_for_tiles(long tiles) { return (int)(tiles < 152L * 16 ? (tiles < 1 ? 1 : tiles) : 152L * 16); }

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_apply_full_fibres(demag_plan* P, const float* m, float* phi, void* stream) {
  demag_status s = check_fft_plan(P, "demag_apply_full_fibres");
  if (s != DEMAG_OK) return s;
  if (!m || !phi) return set_error(P, DEMAG_EINVAL, "demag_apply_full_fibres: NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  const long N = (long)n1 * n2 * n3, vol = 3L * M * N;
  if ((long)M * 3 * n1 * n2 > INT_MAX || (long)M * 3 * n3 * n1 > INT_MAX || 3L * n2 * n3 > INT_MAX)
    return set_error(P, DEMAG_EUNSUPPORTED, "demag_apply_full_fibres: too many fibres for one launch");
  if (!P->fib_ws) DEMAG_CUDA(P, cudaMalloc(&P->fib_ws, sizeof(float) * 2 * (size_t)vol));
  float* Y = P->fib_ws;
  float* Z = Y + vol;
  // axis 1, every node: Y[k][q][i3][i2][i1]
  ToepAxis a{};
  a.axis = 0;
  a.rcols = n2 * n3;
  a.ncols = 3 * a.rcols;
  a.in = m;
  a.in_qstride = N;
  a.out = Y;
  s = run_axes(P, &a, 1, "toeplitz_fft_kernel (fibres, axis 1)", st);
  if (s != DEMAG_OK) return s;
  // Z[k][q][i3][i1][i2]
  {
    const long B = 3L * M * n3;
    const long tiles = B * ((n2 + 31) / 32) * ((n1 + 31) / 32);
    DEMAG_LAUNCH(P, kFamMisc, st, transpose_batched_kernel<<<grid_for_tiles(tiles), 256, 0, st>>>(B, n2, n1, Y, Z));
    DEMAG_LAUNCHED(P, "transpose_batched_kernel");
  }
  // axis 2, node k on volume k: Y[k][q][i3][i1][i2]
  ToepAxis b{};
  b.axis = 1;
  b.rcols = n3 * n1;
  b.ncols = M * 3 * b.rcols;
  b.in = Z;
  b.in_bstride = 3 * N;
  b.in_qstride = N;
  b.out = Y;
  b.out_bstride = 3 * N;
  s = run_axes(P, &b, 1, "toeplitz_fft_kernel (fibres, axis 2)", st, nullptr, 2, 1);
  if (s != DEMAG_OK) return s;
  // Z[k][q][i1][i2][i3]
  {
    const long B = 3L * M;
    const long tiles = B * ((n3 + 31) / 32) * (((long)n1 * n2 + 31) / 32);
    DEMAG_LAUNCH(P, kFamMisc, st,
                 transpose_batched_kernel<<<grid_for_tiles(tiles), 256, 0, st>>>(B, n3, n1 * n2, Y, Z));
    DEMAG_LAUNCHED(P, "transpose_batched_kernel");
  }
  // axis 3, node k on volume k: Y[k][q][i1][i2][i3]
  ToepAxis c{};
  c.axis = 2;
  c.rcols = n1 * n2;
  c.ncols = M * 3 * c.rcols;
  c.in = Z;
  c.in_bstride = 3 * N;
  c.in_qstride = N;
  c.out = Y;
  c.out_bstride = 3 * N;
  s = run_axes(P, &c, 1, "toeplitz_fft_kernel (fibres, axis 3)", st, nullptr, 2, 1);
  if (s != DEMAG_OK) return s;
  {
    const long tiles = (long)n2 * ((n1 + 31) / 32) * ((n3 + 31) / 32);
    DEMAG_LAUNCH(P, kFamMisc, st,
                 fibre_sum_kernel<<<grid_for_tiles(tiles), 256, 0, st>>>(M, n1, n2, n3, P->scale, Y, phi));
    DEMAG_LAUNCHED(P, "fibre_sum_kernel");
  }
  return DEMAG_OK;
}

extern "C" demag_status demag_apply_cp_batched(demag_plan* P, int batch, int r, const float* lambda,
                                               const float* U, float* out_w, float* out_U, void* stream) {
  demag_status s = check_fft_plan(P, "demag_apply_cp");
  if (s != DEMAG_OK) return s;
  if (batch < 1 || r < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_cp: batch and r must be >= 1");
  if (!lambda || !U || !out_w || !out_U) return set_error(P, DEMAG_EINVAL, "demag_apply_cp: NULL pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const long nsum = (long)P->n[0] + P->n[1] + P->n[2];
  ToepAxis ax[3];
  long aoff = 0;
  for (int p = 0; p < 3; ++p) {
    ToepAxis& a = ax[p];
    a = ToepAxis{};
    a.axis = p;
    a.rcols = r;
    a.ncols = batch * 3 * r;
    a.in = U + (long)r * aoff;
    a.in_bstride = 3L * r * nsum;
    a.in_qstride = (long)r * nsum;
    a.out = out_U + (long)P->M * 3 * r * aoff;
    a.out_bstride = (long)P->M * 3 * r * nsum;
    aoff += P->n[p];
  }
  s = run_axes(P, ax, 3, "toeplitz_fft_kernel (cp)", st);
  if (s != DEMAG_OK) return s;
  return launch_weights(P, batch, r, lambda, out_w, st);
}

extern "C" demag_status demag_apply_cp(demag_plan* P, int r, const float* lambda, const float* U,
                                       float* out_w, float* out_U, void* stream) {
  return demag_apply_cp_batched(P, 1, r, lambda, U, out_w, out_U, stream);
}

extern "C" demag_status demag_apply_tucker_batched(demag_plan* P, int batch, const int r[3], const float* V,
                                                   float* out_w, float* out_V, void* stream) {
  demag_status s = check_fft_plan(P, "demag_apply_tucker");
  if (s != DEMAG_OK) return s;
  if (batch < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tucker: batch must be >= 1");
  if (!r || !V || !out_w || !out_V) return set_error(P, DEMAG_EINVAL, "demag_apply_tucker: NULL pointer");
  for (int p = 0; p < 3; ++p)
    if (r[p] < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tucker: r[%d] must be >= 1", p);
  cudaStream_t st = (cudaStream_t)stream;
  long qstride = 0;
  for (int p = 0; p < 3; ++p) qstride += (long)r[p] * P->n[p];
  ToepAxis ax[3];
  long aoff = 0;
  for (int p = 0; p < 3; ++p) {
    ToepAxis& a = ax[p];
    a = ToepAxis{};
    a.axis = p;
    a.rcols = r[p];
    a.ncols = batch * 3 * r[p];
    a.in = V + aoff;
    a.in_bstride = 3 * qstride;
    a.in_qstride = qstride;
    a.out = out_V + (long)P->M * 3 * aoff;
    a.out_bstride = (long)P->M * 3 * qstride;
    aoff += (long)r[p] * P->n[p];
  }
  s = run_axes(P, ax, 3, "toeplitz_fft_kernel (tucker)", st);
  if (s != DEMAG_OK) return s;
  return launch_weights(P, batch, 1, nullptr, out_w, st);
}

// Alg. 2 with the compressed kernels of demag_compress_kernel: factors
// W^(q,p)[:, (i, l)] = T(U_p^(q)[:, i]) V^(q,p)[:, l] through the circulant FFT
// kernel with the per-component symbol sets, and cores C^(q) (x) G^(q).
extern "C" demag_status demag_apply_tucker_compressed(demag_plan* P, int batch, const int r[3], const float* core,
                                                      const float* V, float* out_core, float* out_V, void* stream) {
  demag_status s = check_fft_plan(P, "demag_apply_tucker_compressed");
  if (s != DEMAG_OK) return s;
  if (batch < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tucker_compressed: batch must be >= 1");
  if (!r || !V || !out_V || (out_core && !core))
    return set_error(P, DEMAG_EINVAL, "demag_apply_tucker_compressed: NULL pointer");
  for (int p = 0; p < 3; ++p)
    if (r[p] < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tucker_compressed: r[%d] must be >= 1", p);
  CompressedView cv;
  if (!compressed_view(P, &cv))
    return set_error(P, DEMAG_EINVAL, "demag_apply_tucker_compressed: no compressed kernel (demag_compress_kernel)");
  cudaStream_t st = (cudaStream_t)stream;
  long qstride = 0, ostride = 0;
  for (int p = 0; p < 3; ++p) {
    qstride += (long)r[p] * P->n[p];
    ostride += 3L * cv.rho[p] * r[p] * P->n[p];
  }
  ToepAxis ax[3];
  long aoff = 0, ooff = 0;
  for (int p = 0; p < 3; ++p) {
    ToepAxis& a = ax[p];
    a = ToepAxis{};
    a.axis = p;
    a.rcols = r[p];
    a.ncols = batch * 3 * r[p];
    a.in = V + aoff;
    a.in_bstride = 3 * qstride;
    a.in_qstride = qstride;
    a.out = out_V + ooff;
    a.out_bstride = ostride;
    a.kmax = cv.rho[p];
    aoff += (long)r[p] * P->n[p];
    ooff += 3L * cv.rho[p] * r[p] * P->n[p];
  }
  s = run_axes(P, ax, 3, "toeplitz_fft_kernel (compressed tucker)", st, cv.cpair, 3);
  if (s != DEMAG_OK || !out_core) return s;
  return launch_core_kron(P, batch, r, core, out_core, st);
}

extern "C" demag_status demag_apply_tucker(demag_plan* P, const int r[3], const float* V, float* out_w,
                                           float* out_V, void* stream) {
  return demag_apply_tucker_batched(P, 1, r, V, out_w, out_V, stream);
}

extern "C" demag_status demag_apply_tt_batched(demag_plan* P, int batch, const int r[2], const float* G1,
                                               const float* G2, const float* G3, float* out_w, float* oG1,
                                               float* oG2, float* oG3, void* stream) {
  demag_status s = check_fft_plan(P, "demag_apply_tt");
  if (s != DEMAG_OK) return s;
  if (batch < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tt: batch must be >= 1");
  if (!r || !G1 || !G2 || !G3 || !out_w || !oG1 || !oG2 || !oG3)
    return set_error(P, DEMAG_EINVAL, "demag_apply_tt: NULL pointer");
  if (r[0] < 1 || r[1] < 1) return set_error(P, DEMAG_EINVAL, "demag_apply_tt: TT ranks must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  const int rc[3] = {r[0], r[0] * r[1], r[1]};
  const float* ins[3] = {G1, G2, G3};
  float* outs[3] = {oG1, oG2, oG3};
  ToepAxis ax[3];
  for (int p = 0; p < 3; ++p) {
    ToepAxis& a = ax[p];
    a = ToepAxis{};
    a.axis = p;
    a.rcols = rc[p];
    a.ncols = batch * 3 * rc[p];
    a.in = ins[p];
    a.in_qstride = (long)rc[p] * P->n[p];
    a.in_bstride = 3 * a.in_qstride;
    a.out = outs[p];
    a.out_bstride = (long)P->M * 3 * a.in_qstride;
  }
  s = run_axes(P, ax, 3, "toeplitz_fft_kernel (tt)", st);
  if (s != DEMAG_OK) return s;
  return launch_weights(P, batch, 1, nullptr, out_w, st);
}

extern "C" demag_status demag_apply_tt(demag_plan* P, const int r[2], const float* G1, const float* G2,
                                       const float* G3, float* out_w, float* oG1, float* oG2, float* oG3,
                                       void* stream) {
  return demag_apply_tt_batched(P, 1, r, G1, G2, G3, out_w, oG1, oG2, oG3, stream);
}
