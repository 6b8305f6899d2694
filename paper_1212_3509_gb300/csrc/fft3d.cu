// The potential of a full tensor by one 3D FFT convolution with a dense
// Fourier kernel (Sec. 4.2, Eq. conv_op, Eq. conv_pot, Eq. fft_pot).
//
// P^(q) is a convolution with the separable kernel G^(q)[J], |J_p| < n_p, so
// on a grid padded to L_p >= 2 n_p - 1 per axis (the power of two of the
// plan) phi = IDFT( sum_q K^(q) . DFT(m^(q)) ).  The node sum of
// Eq. conv_pot is linear, so it is summed once per plan into
//
//   K^(q)[w] = c s / (L1 L2 L3) sum_k omega_k prod_p S_{k,q,p}[w_p],
//
// S the DFT of the circulant embedding of the generator F (p == q, odd,
// purely imaginary spectrum) or E (p != q, even, real spectrum).  Hence K^(q)
// is i times a real array, odd in w_q and even in the other frequencies: the
// plan keeps only its imaginary part on the octant 0 <= w_p <= L_p/2
// (FP64 sums rounded once to FP32).  The cost of an application is then
// independent of R.
//
// An application is five passes of batched shared-memory FFTs over fibres;
// each pass reads contiguous fibres and writes its result transposed, so the
// next pass again reads contiguous fibres (index order slowest -> fastest):
//   P1  m[c][i3][i2][i1]    real FFT along i1 (two fibres per complex FFT)
//       -> S1[c][w1][i3][i2]  (w1 <= L1/2)
//   P2  FFT along i2 (zero-padded)   -> S2[c][w2][w1][i3]
//   P3  FFT along i3 (zero-padded), times K^(c), summed over c, inverse FFT
//       along w3, kept i3 < n3      -> S3[i3][w1][w2]   (aliases S1)
//   P4  inverse FFT along w2, kept i2 < n2 -> S4[i2][i3][w1]   (aliases S2)
//   P5  inverse real FFT along w1 (two fibres per complex FFT) -> phi[i3][i2][i1]
// All arithmetic after the FP64 kernel setup is FP32.
//
// The stray field of the analytic derivative factors runs the same passes with
// six real kernels K_pq (h_d[p] = sum_q K_pq * m^(q)): the axis-3 pass then
// transforms the three components, multiplies each bin by the 3 x 3 kernel
// and inverse-transforms three outputs, and P4 / P5 run over three components.
#include <algorithm>
#include <cmath>
#include <new>

#include "fft.cuh"
#include "internal.h"

namespace demag {

constexpr int kFft3dMaxLog = 11;  // L_p <= 2048 (n_p <= 1024)

// Launch shape for an FFT of length N = 2^LOGN along one axis: TG threads
// per fibre, G fibres per block (at least 16, so that the transposed stores
// write runs of >= 128 bytes), buffers padded by pad16 and separated by an
// odd stride so that the same bin of different fibres falls in different banks.
// N = 2048 takes 128 threads (four warps, 16 bins each) per fibre and 4
// fibres per block (register and shared-memory budget); its groups
// synchronise the block.
constexpr int f3_tg(int N) { return N >= 2048 ? 128 : (N / 16 < 1 ? 1 : (N / 16 > 32 ? 32 : N / 16)); }
constexpr int f3_fibres(int N) { return N >= 2048 ? 4 : (16 * f3_tg(N) < 256 ? 256 / f3_tg(N) : 16); }
constexpr int f3_block(int N) { return f3_fibres(N) * f3_tg(N); }
// P3 double-buffers its fibres: half the fibres per block for N = 512 and
// 1024 (two blocks of 256 threads per SM at 128 registers instead of one of
// 512); N = 2048 keeps its 4 fibres (512 threads, one block per SM)
constexpr int f3_fibres_p3(int N) {
  return N >= 2048 ? f3_fibres(N) : (N >= 512 ? f3_fibres(N) / 2 : f3_fibres(N));
}

template <int LOGN> struct F3 {
  static constexpr int N = 1 << LOGN;
  static constexpr int R1 = LOGN < 4 ? N : ((LOGN % 4) ? (1 << (LOGN % 4)) : 16);
  static constexpr int NPASS = LOGN < 4 ? 1 : 1 + (LOGN - (LOGN % 4 ? LOGN % 4 : 4)) / 4;
  static constexpr int TG = f3_tg(N);
  static constexpr int BLOCK = f3_block(N);
  static constexpr int G = f3_fibres(N);
  static constexpr int BS = N + N / 16 + 1;  // per-fibre buffer stride (odd)
  static constexpr size_t smem = ((size_t)N + (size_t)G * BS) * sizeof(float2);
  static constexpr int G3 = f3_fibres_p3(N);  // P3: fibres per block, two buffers each
  static constexpr int BLOCK3 = G3 * TG;
  static constexpr size_t smem3 = ((size_t)N + (size_t)2 * G3 * BS) * sizeof(float2);
  static constexpr size_t smem3f = ((size_t)N + (size_t)3 * G3 * BS) * sizeof(float2);  // field: 3 spectra
  static constexpr int PER = N / TG;  // bins per thread of its fibre
  // N = 2^(4j+1): the radix-2 pass is skipped on zero-padded input (forward)
  // and folded into the reader of the first N/2 outputs (inverse)
  static constexpr bool FOLD = LOGN >= 5 && LOGN % 4 == 1;
  static constexpr int SL = FOLD ? N / 2 : N;  // staged length of a forward input
};

// Synchronise the threads of one FFT group: a warp when the group lies inside
// one (TG <= 32), else the block (all groups run the same code in lockstep).
template <int TG>
__device__ __forceinline__ void group_sync() {
  if constexpr (TG > 32)
    __syncthreads();
  else
    __syncwarp();
}

// In-place complex FFT of length N on a pad16-indexed buffer by the TG
// threads of one group (Stockham, natural order in and out).  First a pass
// of radix R1 (no twiddles), then radix-16 passes.  tw[m] = exp(-2 pi i m / N).
// A group lies inside one warp (TG <= 32), so the passes synchronise the
// warp only; every lane of the warp must call it.
template <int LOGN, bool INV>
__device__ __forceinline__ void fft_pad(float2* buf, int lt, const float2* tw) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, R1 = C::R1;
  {
    constexpr int items = N / R1;
    constexpr int ipt = (items + TG - 1) / TG;
    float2 v[ipt][R1];
#pragma unroll
    for (int it = 0; it < ipt; ++it) {
      const int j = lt + it * TG;
      if (items % TG == 0 || j < items) {
#pragma unroll
        for (int r = 0; r < R1; ++r) v[it][r] = buf[pad16(j + r * items)];
        dft_reg<R1, INV>(v[it]);
      }
    }
    group_sync<TG>();
#pragma unroll
    for (int it = 0; it < ipt; ++it) {
      const int j = lt + it * TG;
      if (items % TG == 0 || j < items) {
#pragma unroll
        for (int r = 0; r < R1; ++r) buf[pad16(j * R1 + r)] = v[it][r];
      }
    }
    group_sync<TG>();
  }
  if constexpr (C::NPASS > 1) {
    int Ns = R1;
#pragma unroll
    for (int ps = 1; ps < C::NPASS; ++ps) {
      constexpr int items = N / 16;
      constexpr int ipt = (items + TG - 1) / TG;
      float2 v[ipt][16];
#pragma unroll
      for (int it = 0; it < ipt; ++it) {
        const int j = lt + it * TG;
        if (items % TG == 0 || j < items) {
          const int k = j % Ns;
          float2 w = tw[k * (N / (Ns * 16))];
          if (INV) w.y = -w.y;
          float2 pw[16];
          powers<16>(w, pw);
#pragma unroll
          for (int r = 0; r < 16; ++r) {
            const float2 x = buf[pad16(j + r * items)];
            v[it][r] = r > 0 ? cmul(x, pw[r]) : x;
          }
          dft_reg<16, INV>(v[it]);
        }
      }
      group_sync<TG>();
#pragma unroll
      for (int it = 0; it < ipt; ++it) {
        const int j = lt + it * TG;
        if (items % TG == 0 || j < items) {
          const int k = j % Ns;
          const int base = (j / Ns) * Ns * 16 + k;
#pragma unroll
          for (int r = 0; r < 16; ++r) buf[pad16(base + r * Ns)] = v[it][r];
        }
      }
      group_sync<TG>();
      Ns *= 16;
    }
  }
}

// One in-place radix-16 Stockham pass over sub-transforms of size Ns.  With
// DUP the pass input is y[m] = x[m >> 1]: the output of a radix-2 first pass
// on an input with x[j] = 0 for j >= N/2, which only duplicates
// (y[2j] = y[2j+1] = x[j]) and is therefore not done.
template <int LOGN, bool INV, bool DUP>
__device__ __forceinline__ void r16_pass(float2* buf, int Ns, int lt, const float2* tw) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG;
  constexpr int items = N / 16;
  constexpr int ipt = (items + TG - 1) / TG;
  float2 v[ipt][16];
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        // pad16(i + r S) = pad16(i) + r (S + S/16) when S is a multiple of 16
        if constexpr (DUP && (items / 2) % 16 == 0)
          v[it][r] = buf[pad16(j >> 1) + r * PadStride<items / 2>::value];
        else if constexpr (!DUP && items % 16 == 0)
          v[it][r] = buf[pad16(j) + r * PadStride<items>::value];
        else
          v[it][r] = buf[pad16(DUP ? ((j + r * items) >> 1) : (j + r * items))];
      }
      if (Ns > 1) {  // (Ns = 1: all twiddles are 1)
        float2 w = tw[k * (N / (Ns * 16))];
        if (INV) w.y = -w.y;
        float2 pw[16];
        powers<16>(w, pw);
#pragma unroll
        for (int r = 1; r < 16; ++r) v[it][r] = cmul(v[it][r], pw[r]);
      }
      dft_reg<16, INV>(v[it]);
    }
  }
  group_sync<TG>();
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * 16 + k;
      if (Ns % 16 == 0) {
        const int b0 = pad16(base), step = Ns + (Ns >> 4);
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[b0 + r * step] = v[it][r];
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) buf[pad16(base + r * Ns)] = v[it][r];
      }
    }
  }
  group_sync<TG>();
}

// Forward FFT of a fibre staged in its first SL slots (zeros past the data).
template <int LOGN>
__device__ __forceinline__ void fwd_fft(float2* buf, int lt, const float2* tw) {
  using C = F3<LOGN>;
  if constexpr (C::FOLD) {
    r16_pass<LOGN, false, true>(buf, 2, lt, tw);
#pragma unroll
    for (int ps = 2, Ns = 32; ps < C::NPASS; ++ps, Ns *= 16) r16_pass<LOGN, false, false>(buf, Ns, lt, tw);
  } else {
    fft_pad<LOGN, false>(buf, lt, tw);
  }
}

// Inverse FFT whose outputs k < N/2 are then read with inv_out (with FOLD the
// last radix-2 pass is left to inv_out).
template <int LOGN>
__device__ __forceinline__ void inv_fft(float2* buf, int lt, const float2* tw) {
  using C = F3<LOGN>;
  if constexpr (C::FOLD) {
#pragma unroll
    for (int ps = 1, Ns = 1; ps < C::NPASS; ++ps, Ns *= 16) r16_pass<LOGN, true, false>(buf, Ns, lt, tw);
  } else {
    fft_pad<LOGN, true>(buf, lt, tw);
  }
}

// Output k < N/2 of inv_fft: with FOLD the last radix-2 butterfly (Ns = N/2)
// y_k = x_k + conj(W_N^k) x_{k + N/2}.
template <int LOGN>
__device__ __forceinline__ float2 inv_out(const float2* buf, int k, const float2* tw) {
  using C = F3<LOGN>;
  if constexpr (C::FOLD) {
    float2 w = tw[k];
    w.y = -w.y;
    const float2 a = buf[pad16(k)], b = buf[pad16(k + C::N / 2)];
    return cadd(a, cmul(b, w));
  } else {
    return buf[pad16(k)];
  }
}

struct Fft3dArgs {
  int n1, n2, n3;
  int L1, L2, L3;
  int H1, H2, H3;         // L_p / 2 + 1
  const float* m;         // [3][n3][n2][n1]
  float2* s1;             // [3][H1][n3][n2]; S3 [n3][H1][L2] aliases it
  float2* s2;             // [3][L2][H1][n3]; S4 [n2][n3][H1] aliases it
  float* phi;             // [n3][n2][n1]
  const float* kst;       // [3][H1][H2][H3]: Im K^(q) on the octant
  const float* kfield;    // [6][H1][H2][H3]: the real field kernels K_pq on the octant (pairs 00 11 22 01 02 12)
  const float2* tw;       // exp(-2 pi i m / N) of this pass's axis, m < N
  int nco;                // components after P3: 1 (potential) or 3 (field)
};

template <int LOGN>
__device__ __forceinline__ void load_twiddles(float2* tw, const float2* src) {
  for (int i = threadIdx.x; i < (1 << LOGN); i += blockDim.x) tw[i] = __ldg(src + i);
}

// Fibre in[0..n) zero-padded to N into the pad16-indexed buffer; every load
// is issued before the first shared-memory store.
template <int LOGN, int LEN>
__device__ __forceinline__ void stage_fibre(float2* buf, int lt, const float2* in, int n) {
  using C = F3<LOGN>;
  constexpr int CNT = (LEN + C::TG - 1) / C::TG;
  float2 ld[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int j = lt + i * C::TG;
    ld[i] = j < n ? __ldg(in + j) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int j = lt + i * C::TG;
    if (LEN % C::TG == 0 || j < LEN) buf[pad16(j)] = ld[i];
  }
}

// cp.async of one float2 into shared memory; zero-filled (nothing read) when !pred.
__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool pred) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(PENDING) : "memory");
}

// The same fibre copy as stage_fibre, asynchronous (cp.async); `in` must be
// a valid address even when n == 0.
template <int LOGN, int LEN>
__device__ __forceinline__ void copy_fibre_async(float2* buf, int lt, const float2* in, int n) {
  using C = F3<LOGN>;
  constexpr int CNT = (LEN + C::TG - 1) / C::TG;
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int j = lt + i * C::TG;
    if (LEN % C::TG == 0 || j < LEN) cp_async8(buf + pad16(j), j < n ? in + j : in, j < n);
  }
}

// P1: real FFT along i1 of fibre pairs (i2, i2 + 1) at fixed (c, i3).
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK) fft3d_p1_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G, BS = C::BS, T = 2 * G;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  float2* bufs = sm3 + N;
  load_twiddles<LOGN>(tw, a.tw);
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* buf = bufs + g * BS;
  const int tiles = (a.n2 + T - 1) / T;
  const int tile = blockIdx.x % tiles;
  const int ci3 = blockIdx.x / tiles;  // c * n3 + i3
  const int i2a = tile * T + 2 * g;
  const float* row = a.m + (size_t)ci3 * a.n2 * a.n1;
  const bool va = i2a < a.n2, vb = i2a + 1 < a.n2;
  // all loads of the fibre pair in flight before the first shared-memory store
  constexpr int CNT = C::SL / TG;
  float2 ld[CNT];
#pragma unroll
  for (int i = 0; i < CNT; ++i) {
    const int j = lt + i * TG;
    float x = 0.f, y = 0.f;
    if (j < a.n1) {
      if (va) x = __ldg(row + (size_t)i2a * a.n1 + j);
      if (vb) y = __ldg(row + (size_t)(i2a + 1) * a.n1 + j);
    }
    ld[i] = make_float2(x, y);
  }
#pragma unroll
  for (int i = 0; i < CNT; ++i) buf[pad16(lt + i * TG)] = ld[i];
  __syncthreads();
  fwd_fft<LOGN>(buf, lt, tw);
  __syncthreads();  // the split step reads every fibre pair's buffer
  // X_a = (Z_w + conj Z_{N-w}) / 2, X_b = (Z_w - conj Z_{N-w}) / 2i; stored at S1[c][w][i3][i2]
  const int c = ci3 / a.n3, i3 = ci3 % a.n3;
  float2* out = a.s1 + (size_t)c * a.H1 * a.n3 * a.n2 + (size_t)i3 * a.n2 + (size_t)tile * T;
  const int lim = min(T, a.n2 - tile * T);
  auto split = [&](int w, int g2) {
    const float2* b = bufs + (g2 >> 1) * BS;
    const float2 Z = b[pad16(w)], Zc = b[pad16((N - w) & (N - 1))];
    return (g2 & 1) ? make_float2(0.5f * (Z.y + Zc.y), -0.5f * (Z.x - Zc.x))
                    : make_float2(0.5f * (Z.x + Zc.x), 0.5f * (Z.y - Zc.y));
  };
  if constexpr (C::BLOCK % T == 0) {
    // thread -> fibre g2 = tid % T (fixed), rows w = tid / T + k (BLOCK / T)
    constexpr int WS = C::BLOCK / T;
    const int g2 = threadIdx.x % T;
    if (g2 < lim) {
      const size_t step = (size_t)WS * a.n3 * a.n2;
      float2* dst = out + g2 + (size_t)(threadIdx.x / T) * a.n3 * a.n2;
#pragma unroll 4
      for (int w = threadIdx.x / T; w < a.H1; w += WS, dst += step) *dst = split(w, g2);
    }
  } else {
    for (int idx = threadIdx.x; idx < a.H1 * T; idx += C::BLOCK) {
      const int w = idx / T, g2 = idx % T;
      if (g2 < lim) out[(size_t)w * a.n3 * a.n2 + g2] = split(w, g2);
    }
  }
}

// P2: FFT along i2 (n2 samples zero-padded to L2) of fibres i3 at fixed (c, w1).
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK) fft3d_p2_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G, BS = C::BS;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  float2* bufs = sm3 + N;
  load_twiddles<LOGN>(tw, a.tw);
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* buf = bufs + g * BS;
  const int tiles = (a.n3 + G - 1) / G;
  const int tile = blockIdx.x % tiles;
  const int cw1 = blockIdx.x / tiles;  // c * H1 + w1
  const int i3 = tile * G + g;
  const float2* in = a.s1 + ((size_t)cw1 * a.n3 + i3) * a.n2;
  stage_fibre<LOGN, C::SL>(buf, lt, in, i3 < a.n3 ? a.n2 : 0);
  __syncthreads();
  fwd_fft<LOGN>(buf, lt, tw);
  __syncthreads();  // the transposed store reads every fibre's buffer
  const int c = cw1 / a.H1, w1 = cw1 % a.H1;
  float2* out = a.s2 + (size_t)c * a.L2 * a.H1 * a.n3 + (size_t)w1 * a.n3 + (size_t)tile * G;
  const int lim = min(G, a.n3 - tile * G);
  // thread -> fibre gg = tid % G (fixed), rows w2 = tid / G + k TG
  const int gg = threadIdx.x % G;
  if (gg < lim) {
    const float2* src = bufs + gg * BS;
    const size_t step = (size_t)TG * a.H1 * a.n3;
    float2* dst = out + gg + (size_t)(threadIdx.x / G) * a.H1 * a.n3;
#pragma unroll 4
    for (int w2 = threadIdx.x / G; w2 < N; w2 += TG, dst += step) *dst = src[pad16(w2)];
  }
}

// P3: at fixed w1, fibres w2 along i3: forward FFT of each component,
// times K^(c), summed over c in registers, inverse FFT, i3 < n3 kept.  The
// next component's fibres are copied in (cp.async, zero-filled past n3) into
// a second buffer while the current one is transformed.
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK3, LOGN <= 9 ? 2 : 1) fft3d_p3_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G3, BS = C::BS, PER = C::PER;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* bufc[2] = {sm3 + N + g * BS, sm3 + N + (G + g) * BS};
  const int tiles = (a.L2 + G - 1) / G;
  const int tile = blockIdx.x % tiles;
  const int w1 = blockIdx.x / tiles;
  const int w2 = tile * G + g;
  const bool valid = w2 < a.L2;
  const int w2f = w2 <= a.L2 / 2 ? w2 : a.L2 - w2;
  const int nload = valid ? a.n3 : 0;
  auto fibre = [&](int c) { return a.s2 + (((size_t)c * a.L2 + (valid ? w2 : 0)) * a.H1 + w1) * a.n3; };
  copy_fibre_async<LOGN, C::SL>(bufc[0], lt, fibre(0), nload);
  cp_async_commit();
  load_twiddles<LOGN>(tw, a.tw);
  float2 acc[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2* buf = bufc[c & 1];
    if (c < 2) {
      copy_fibre_async<LOGN, C::SL>(bufc[(c + 1) & 1], lt, fibre(c + 1), nload);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    // the fibre's copies were issued by its own warp; the twiddle table by the block
    if (c == 0)
      __syncthreads();
    else
      group_sync<TG>();
    fwd_fft<LOGN>(buf, lt, tw);
    const float* krow = a.kst + (((size_t)c * a.H1 + w1) * a.H2 + (valid ? w2f : 0)) * a.H3;
    const float s2sign = (c == 1 && w2 > a.L2 / 2) ? -1.f : 1.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int w3 = lt + j * TG;
      const int w3f = w3 <= N / 2 ? w3 : N - w3;
      float kv = __ldg(krow + w3f) * s2sign;
      if (c == 2 && w3 > N / 2) kv = -kv;
      const float2 Z = buf[pad16(w3)];
      // (i kv) Z
      acc[j].x = fmaf(-kv, Z.y, acc[j].x);
      acc[j].y = fmaf(kv, Z.x, acc[j].y);
    }
    group_sync<TG>();
  }
  float2* buf = bufc[0];
#pragma unroll
  for (int j = 0; j < PER; ++j) buf[pad16(lt + j * TG)] = acc[j];
  group_sync<TG>();
  inv_fft<LOGN>(buf, lt, tw);
  __syncthreads();  // the transposed store reads every fibre's buffer
  float2* out = a.s1 + (size_t)w1 * a.L2 + (size_t)tile * G;  // S3[i3][w1][w2]
  const int lim = min(G, a.L2 - tile * G);
  const float2* bufs = sm3 + N;
  const int gg = threadIdx.x % G;
  if (gg < lim) {
    const float2* src = bufs + gg * BS;
    const size_t step = (size_t)TG * a.H1 * a.L2;
    float2* dst = out + gg + (size_t)(threadIdx.x / G) * a.H1 * a.L2;
#pragma unroll 4
    for (int i3 = threadIdx.x / G; i3 < a.n3; i3 += TG, dst += step) *dst = inv_out<LOGN>(src, i3, tw);
  }
}

// P3 of the stray field: at fixed w1, fibres w2 along i3: forward FFT of the
// three components (all three copied in at once, cp.async), then per bin
// Y_p = sum_q K_pq X_q with the real, symmetric field kernels (in place: a
// bin of Y needs only the same bin of the X), inverse FFTs, i3 < n3 kept, into
// S3[p][i3][w1][w2].  K_pq is odd in w_p and w_q for p != q and even
// otherwise, so the octant value takes a sign for each mirrored odd axis.
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK3, LOGN <= 9 ? 2 : 1) fft3d_p3f_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G3, BS = C::BS, PER = C::PER;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* bq[3] = {sm3 + N + g * BS, sm3 + N + (G + g) * BS, sm3 + N + (2 * G + g) * BS};
  const int tiles = (a.L2 + G - 1) / G;
  const int tile = blockIdx.x % tiles;
  const int w1 = blockIdx.x / tiles;
  const int w2 = tile * G + g;
  const bool valid = w2 < a.L2;
  const bool m2 = w2 > a.L2 / 2;
  const int w2f = m2 ? a.L2 - w2 : w2;
  const int nload = valid ? a.n3 : 0;
#pragma unroll
  for (int c = 0; c < 3; ++c)
    copy_fibre_async<LOGN, C::SL>(bq[c], lt, a.s2 + (((size_t)c * a.L2 + (valid ? w2 : 0)) * a.H1 + w1) * a.n3, nload);
  cp_async_commit();
  load_twiddles<LOGN>(tw, a.tw);
  cp_async_wait<0>();
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) fwd_fft<LOGN>(bq[c], lt, tw);
  const size_t oct = (size_t)a.H1 * a.H2 * a.H3;
  const float* krow = a.kfield + ((size_t)w1 * a.H2 + (valid ? w2f : 0)) * a.H3;
#pragma unroll 4
  for (int j = 0; j < PER; ++j) {
    const int w3 = lt + j * TG;
    const bool m3 = w3 > N / 2;
    const int w3f = m3 ? N - w3 : w3;
    const float k00 = __ldg(krow + w3f), k11 = __ldg(krow + oct + w3f), k22 = __ldg(krow + 2 * oct + w3f);
    float k01 = __ldg(krow + 3 * oct + w3f), k02 = __ldg(krow + 4 * oct + w3f), k12 = __ldg(krow + 5 * oct + w3f);
    if (m2) {
      k01 = -k01;
      k12 = -k12;
    }
    if (m3) {
      k02 = -k02;
      k12 = -k12;
    }
    const int b = pad16(w3);
    const float2 x0 = bq[0][b], x1 = bq[1][b], x2 = bq[2][b];
    bq[0][b] = make_float2(k00 * x0.x + k01 * x1.x + k02 * x2.x, k00 * x0.y + k01 * x1.y + k02 * x2.y);
    bq[1][b] = make_float2(k01 * x0.x + k11 * x1.x + k12 * x2.x, k01 * x0.y + k11 * x1.y + k12 * x2.y);
    bq[2][b] = make_float2(k02 * x0.x + k12 * x1.x + k22 * x2.x, k02 * x0.y + k12 * x1.y + k22 * x2.y);
  }
  group_sync<TG>();
#pragma unroll
  for (int c = 0; c < 3; ++c) inv_fft<LOGN>(bq[c], lt, tw);
  __syncthreads();  // the transposed stores read every fibre's buffers
  const int lim = min(G, a.L2 - tile * G);
  const int gg = threadIdx.x % G;
  if (gg < lim) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2* src = sm3 + N + (c * G + gg) * BS;
      const size_t step = (size_t)TG * a.H1 * a.L2;
      float2* dst = a.s1 + (size_t)c * a.n3 * a.H1 * a.L2 + (size_t)w1 * a.L2 + (size_t)tile * G + gg +
                    (size_t)(threadIdx.x / G) * a.H1 * a.L2;
      for (int i3 = threadIdx.x / G; i3 < a.n3; i3 += TG, dst += step) *dst = inv_out<LOGN>(src, i3, tw);
    }
  }
}

// P4: inverse FFT along w2 of fibres w1 at fixed (c, i3), i2 < n2 kept.
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK) fft3d_p4_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G, BS = C::BS;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  float2* bufs = sm3 + N;
  load_twiddles<LOGN>(tw, a.tw);
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* buf = bufs + g * BS;
  const int tiles = (a.H1 + G - 1) / G;
  const int tile = blockIdx.x % tiles;
  const int ci3 = blockIdx.x / tiles;  // c * n3 + i3
  const int c = ci3 / a.n3, i3 = ci3 % a.n3;
  const int w1 = tile * G + g;
  const float2* in = a.s1 + (size_t)c * a.n3 * a.H1 * a.L2 + ((size_t)i3 * a.H1 + w1) * a.L2;
  stage_fibre<LOGN, N>(buf, lt, in, w1 < a.H1 ? N : 0);
  __syncthreads();
  inv_fft<LOGN>(buf, lt, tw);
  __syncthreads();  // the transposed store reads every fibre's buffer
  float2* out = a.s2 + (size_t)c * a.n2 * a.n3 * a.H1 + (size_t)i3 * a.H1 + (size_t)tile * G;  // S4[c][i2][i3][w1]
  const int lim = min(G, a.H1 - tile * G);
  const int gg = threadIdx.x % G;
  if (gg < lim) {
    const float2* src = bufs + gg * BS;
    const size_t step = (size_t)TG * a.n3 * a.H1;
    float2* dst = out + gg + (size_t)(threadIdx.x / G) * a.n3 * a.H1;
#pragma unroll 4
    for (int i2 = threadIdx.x / G; i2 < a.n2; i2 += TG, dst += step) *dst = inv_out<LOGN>(src, i2, tw);
  }
}

// P5: inverse real FFT along w1 of fibre pairs f, f + 1 (f = (c n2 + i2) n3 + i3).
template <int LOGN>
__global__ void __launch_bounds__(F3<LOGN>::BLOCK) fft3d_p5_kernel(const __grid_constant__ Fft3dArgs a) {
  using C = F3<LOGN>;
  constexpr int N = C::N, TG = C::TG, G = C::G, BS = C::BS, T = 2 * G;
  extern __shared__ float2 sm3[];
  float2* tw = sm3;
  float2* bufs = sm3 + N;
  load_twiddles<LOGN>(tw, a.tw);
  const int g = threadIdx.x / TG, lt = threadIdx.x % TG;
  float2* buf = bufs + g * BS;
  const int nf = a.nco * a.n2 * a.n3;
  const int fa = blockIdx.x * T + 2 * g;
  const bool va = fa < nf, vb = fa + 1 < nf;
  const float2* ina = a.s2 + (size_t)fa * a.H1;
  const float2* inb = ina + a.H1;
  const float2 zero = make_float2(0.f, 0.f);
  // two rounds of loads (half the bins each), all of a round in flight before its stores
  constexpr int HALF = C::PER > 1 ? C::PER / 2 : 1;
#pragma unroll
  for (int i0 = 0; i0 < C::PER; i0 += HALF) {
    float2 la[HALF], lb[HALF];
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
      const int w = lt + (i0 + i) * TG;
      const int src = w <= N / 2 ? w : N - w;
      la[i] = va ? __ldg(ina + src) : zero;
      lb[i] = vb ? __ldg(inb + src) : zero;
    }
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
      const int w = lt + (i0 + i) * TG;
      // Hermitian extension X_w = conj X_{N-w}; the imaginary parts at w = 0, N/2 are dropped
      float2 xa = la[i], xb = lb[i];
      if (w > N / 2) {
        xa.y = -xa.y;
        xb.y = -xb.y;
      }
      if (w == 0 || w == N / 2) {
        xa.y = 0.f;
        xb.y = 0.f;
      }
      buf[pad16(w)] = make_float2(xa.x - xb.y, xa.y + xb.x);  // X_a + i X_b
    }
  }
  __syncthreads();
  inv_fft<LOGN>(buf, lt, tw);
  // fibre f = (c n2 + i2) n3 + i3 -> phi[c][i3][i2][:]
  auto row = [&](int f) {
    const int i3 = f % a.n3, ci2 = f / a.n3;
    const int i2 = ci2 % a.n2, c = ci2 / a.n2;
    return a.phi + (((size_t)c * a.n3 + i3) * a.n2 + i2) * a.n1;
  };
  float* oa = row(va ? fa : 0);
  float* ob = row(vb ? fa + 1 : 0);
  for (int j = lt; j < a.n1; j += TG) {
    const float2 v = inv_out<LOGN>(buf, j, tw);
    if (va) oa[j] = v.x;
    if (vb) ob[j] = v.y;
  }
}

// ---------------------------------------------------------------- setup

// sym[k][type][p][w] (w <= L_p/2), FP64: the DFT of the circulant embedding
// of generator row (k, type, p) divided by L_p; an even generator: the real
// part t0 + 2 sum_d t_d cos(2 pi w d / L); the odd one (type odd_type: F of
// the generators, dE of the derivative generators): the imaginary part
// -2 sum_d t_d sin(2 pi w d / L).  Angles are reduced exactly ((w d) mod L).
__global__ void fft3d_symbols_kernel(int M, int glen, int hstride, int n1, int n2, int n3, int L1, int L2, int L3,
                                     const double* gen64, double* sym, int odd_type) {
  const long total = (long)M * 2 * 3 * hstride;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const int w = (int)(idx % hstride);
    long rest = idx / hstride;
    const int p = (int)(rest % 3);
    rest /= 3;
    const int type = (int)(rest % 2);
    const int k = (int)(rest / 2);
    const int n = p == 0 ? n1 : (p == 1 ? n2 : n3);
    const int L = p == 0 ? L1 : (p == 1 ? L2 : L3);
    double val = 0.0;
    if (w <= L / 2) {
      const double* t = gen64 + (((long)k * 2 + type) * 3 + p) * glen + (n - 1);  // t[d], |d| < n
      double acc = 0.0;
      for (int d = 1; d < n; ++d) {
        const int r = (int)(((long)w * d) % L);
        double sn, cs;
        sincospi(2.0 * (double)r / (double)L, &sn, &cs);
        acc += type != odd_type ? t[d] * cs : t[d] * sn;
      }
      val = type != odd_type ? (t[0] + 2.0 * acc) : (-2.0 * acc);
      val /= (double)L;
    }
    sym[idx] = val;
  }
}

// kst[c][w1][w2][w3] = sum_k scale_k S_{k,c,1}[w1] S_{k,c,2}[w2] S_{k,c,3}[w3]
// (FP64 sum, one rounding to FP32); scale_k = c s omega_k.  One block per
// (c, w1, w2), threads over w3.
__global__ void fft3d_kernel_kernel(int M, int hstride, int H1, int H2, int H3, const double* scale,
                                    const double* sym, float* kst) {
  __shared__ double a[kMaxTerms];
  const int w2 = blockIdx.x % H2;
  const int cw1 = blockIdx.x / H2;
  const int w1 = cw1 % H1, c = cw1 / H1;
  const int t1 = c == 0, t2 = c == 1, t3 = c == 2;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    a[k] = scale[k] * sym[(((long)k * 2 + t1) * 3 + 0) * hstride + w1] *
           sym[(((long)k * 2 + t2) * 3 + 1) * hstride + w2];
  __syncthreads();
  float* out = kst + ((size_t)cw1 * H2 + w2) * H3;
  for (int w3 = threadIdx.x; w3 < H3; w3 += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < M; ++k) acc += a[k] * sym[(((long)k * 2 + t3) * 3 + 2) * hstride + w3];
    out[w3] = (float)acc;
  }
}

// kfield[pair][w1][w2][w3] (pairs (d, q) = 00 11 22 01 02 12), the real field
// kernels of h_d[d] = sum_q K_dq * m^(q): every factor of Eq. conv_pot's term k
// with the axis-d factor replaced by its derivative (dE for E, dF for F; the
// derivative generators carry 1/s), summed over k with scale_k = c s omega_k
// (FP64, one rounding).  From the reduced symbols (real part of an even
// factor, imaginary part of an odd one): d == q has no odd factor and the sign
// of h = -grad phi; d != q has two (dE along d, F along q), i^2 = -1, sign +.
__global__ void fft3d_field_kernel_kernel(int M, int hstride, int H1, int H2, int H3, const double* scale,
                                          const double* sym, const double* dsym, float* kf) {
  __shared__ double a[kMaxTerms];
  const int pd[6] = {0, 1, 2, 0, 0, 1}, pq[6] = {0, 1, 2, 1, 2, 2};
  const int w2 = blockIdx.x % H2;
  const int rest = blockIdx.x / H2;
  const int w1 = rest % H1, pair = rest / H1;
  const int d = pd[pair], q = pq[pair];
  auto factor = [&](int k, int axis, int w) {
    const int type = axis == q ? 1 : 0;
    const double* src = axis == d ? dsym : sym;
    return src[(((long)k * 2 + type) * 3 + axis) * hstride + w];
  };
  const double sign = d == q ? -1.0 : 1.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x) a[k] = sign * scale[k] * factor(k, 0, w1) * factor(k, 1, w2);
  __syncthreads();
  float* out = kf + (((size_t)pair * H1 + w1) * H2 + w2) * H3;
  for (int w3 = threadIdx.x; w3 < H3; w3 += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < M; ++k) acc += a[k] * factor(k, 2, w3);
    out[w3] = (float)acc;
  }
}

struct Fft3dState {
  int logL[3];
  float* kst = nullptr;
  float* kfield = nullptr;  // stray-field kernels, built on first use
  float* hfield = nullptr;  // [3][n3][n2][n1] field scratch of the energy
  float2* s1 = nullptr;
  float2* s2 = nullptr;
  size_t s1_elems = 0, s2_elems = 0;
};

static int log2_exact(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

template <int LOGN>
static demag_status launch_pass(demag_plan* P, int pass, const Fft3dArgs& a, int blocks, cudaStream_t st) {
  using C = F3<LOGN>;
  // pass 6 is the P3 of the stray field
  const void* fn = pass == 1 ? (const void*)fft3d_p1_kernel<LOGN>
                 : pass == 2 ? (const void*)fft3d_p2_kernel<LOGN>
                 : pass == 3 ? (const void*)fft3d_p3_kernel<LOGN>
                 : pass == 4 ? (const void*)fft3d_p4_kernel<LOGN>
                 : pass == 5 ? (const void*)fft3d_p5_kernel<LOGN>
                             : (const void*)fft3d_p3f_kernel<LOGN>;
  // the attribute is set on first use per kernel and device (so that later
  // launches, e.g. under stream capture, make no attribute calls)
  static unsigned long long done[7] = {0, 0, 0, 0, 0, 0, 0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  const size_t smem = pass == 3 ? C::smem3 : (pass == 6 ? C::smem3f : C::smem);
  if (smem > 48 * 1024 && !(done[pass] & bit)) {
    DEMAG_CUDA(P, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    done[pass] |= bit;
  }
  switch (pass) {
    case 1: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p1_kernel<LOGN><<<blocks, C::BLOCK, C::smem, st>>>(a)); break;
    case 2: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p2_kernel<LOGN><<<blocks, C::BLOCK, C::smem, st>>>(a)); break;
    case 3: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p3_kernel<LOGN><<<blocks, C::BLOCK3, C::smem3, st>>>(a)); break;
    case 4: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p4_kernel<LOGN><<<blocks, C::BLOCK, C::smem, st>>>(a)); break;
    case 5: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p5_kernel<LOGN><<<blocks, C::BLOCK, C::smem, st>>>(a)); break;
    default: DEMAG_LAUNCH(P, kFamFFT3D, st, fft3d_p3f_kernel<LOGN><<<blocks, C::BLOCK3, C::smem3f, st>>>(a)); break;
  }
  DEMAG_LAUNCHED(P, "fft3d pass");
  return DEMAG_OK;
}

static demag_status dispatch_pass(demag_plan* P, int logn, int pass, const Fft3dArgs& a, int blocks,
                                  cudaStream_t st) {
  switch (logn) {
    case 1: return launch_pass<1>(P, pass, a, blocks, st);
    case 2: return launch_pass<2>(P, pass, a, blocks, st);
    case 3: return launch_pass<3>(P, pass, a, blocks, st);
    case 4: return launch_pass<4>(P, pass, a, blocks, st);
    case 5: return launch_pass<5>(P, pass, a, blocks, st);
    case 6: return launch_pass<6>(P, pass, a, blocks, st);
    case 7: return launch_pass<7>(P, pass, a, blocks, st);
    case 8: return launch_pass<8>(P, pass, a, blocks, st);
    case 9: return launch_pass<9>(P, pass, a, blocks, st);
    case 10: return launch_pass<10>(P, pass, a, blocks, st);
    case 11: return launch_pass<11>(P, pass, a, blocks, st);
    default: return set_error(P, DEMAG_EUNSUPPORTED, "fft3d: FFT length 2^%d not supported", logn);
  }
}

demag_status fft3d_prepare(demag_plan* P, cudaStream_t st) {
  if (P->f3) return DEMAG_OK;
  demag_status u = require_uniform(P, "demag_apply_full_fft");  // a convolution needs Toeplitz factors
  if (u != DEMAG_OK) return u;
  for (int p = 0; p < 3; ++p)
    if (P->L[p] > (1 << kFft3dMaxLog))
      return set_error(P, DEMAG_EUNSUPPORTED, "demag_apply_full_fft: n[%d] = %d exceeds %d", p, P->n[p],
                       (1 << kFft3dMaxLog) / 2);
  if (!P->twid[0] || !P->twid[1] || !P->twid[2])
    return set_error(P, DEMAG_EUNSUPPORTED, "demag_apply_full_fft: plan has no FFT twiddles");
  Fft3dState* S = new (std::nothrow) Fft3dState();
  if (!S) return set_error(P, DEMAG_ENOMEM, "host allocation failed");
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const int L1 = P->L[0], L2 = P->L[1], L3 = P->L[2];
  const int H1 = L1 / 2 + 1, H2 = L2 / 2 + 1, H3 = L3 / 2 + 1;
  for (int p = 0; p < 3; ++p) S->logL[p] = log2_exact(P->L[p]);
  // S1 holds [3][H1][n3][n2] and later S3 [n3][H1][L2]; S2 [3][L2][H1][n3] and later S4 [n2][n3][H1]
  S->s1_elems = std::max((size_t)3 * H1 * n3 * n2, (size_t)n3 * H1 * L2);
  S->s2_elems = std::max((size_t)3 * L2 * H1 * n3, (size_t)n2 * n3 * H1);
  const int hstride = std::max(H1, std::max(H2, H3));
  double* sym = nullptr;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaFree(sym);
    cudaFree(S->kst);
    cudaFree(S->s1);
    cudaFree(S->s2);
    delete S;
    return cuda_error(P, e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&S->kst, sizeof(float) * 3 * (size_t)H1 * H2 * H3)) != cudaSuccess) return fail(e, "malloc kst");
  if ((e = cudaMalloc(&S->s1, sizeof(float2) * S->s1_elems)) != cudaSuccess) return fail(e, "malloc s1");
  if ((e = cudaMalloc(&S->s2, sizeof(float2) * S->s2_elems)) != cudaSuccess) return fail(e, "malloc s2");
  if ((e = cudaMalloc(&sym, sizeof(double) * (size_t)P->M * 6 * hstride)) != cudaSuccess) return fail(e, "malloc sym");
  {
    const long total = (long)P->M * 6 * hstride;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 32) blocks = 152 * 32;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 fft3d_symbols_kernel<<<blocks, 256, 0, st>>>(P->M, P->glen, hstride, n1, n2, n3, L1, L2, L3,
                                                              P->gen64, sym, 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "fft3d_symbols_kernel");
    DEMAG_LAUNCH(P, kFamSetup, st,
                 fft3d_kernel_kernel<<<3 * H1 * H2, 256, 0, st>>>(P->M, hstride, H1, H2, H3, P->scale, sym,
                                                                  S->kst));
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "fft3d_kernel_kernel");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e, "fft3d setup");
  cudaFree(sym);
  P->f3 = S;
  return DEMAG_OK;
}

// The stray-field kernels (once per plan) and room for three components in
// S3 (it aliases S1).
static demag_status fft3d_prepare_field(demag_plan* P, cudaStream_t st) {
  demag_status rc = fft3d_prepare(P, st);
  if (rc != DEMAG_OK) return rc;
  Fft3dState* S = static_cast<Fft3dState*>(P->f3);
  if (S->kfield) return DEMAG_OK;
  rc = ensure_field_generators(P, st);
  if (rc != DEMAG_OK) return rc;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const int L1 = P->L[0], L2 = P->L[1], L3 = P->L[2];
  const int H1 = L1 / 2 + 1, H2 = L2 / 2 + 1, H3 = L3 / 2 + 1;
  const size_t s1_need = std::max(S->s1_elems, (size_t)3 * n3 * H1 * L2);
  if (s1_need > S->s1_elems) {
    DEMAG_CUDA(P, cudaStreamSynchronize(st));
    cudaFree(S->s1);
    S->s1 = nullptr;
    S->s1_elems = 0;
    DEMAG_CUDA(P, cudaMalloc(&S->s1, sizeof(float2) * s1_need));
    S->s1_elems = s1_need;
  }
  const int hstride = std::max(H1, std::max(H2, H3));
  const size_t nsym = (size_t)P->M * 6 * hstride;
  double* sym = nullptr;
  float* kf = nullptr;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaFree(sym);
    cudaFree(kf);
    return cuda_error(P, e, what);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&sym, sizeof(double) * 2 * nsym)) != cudaSuccess) return fail(e, "malloc field symbols");
  if ((e = cudaMalloc(&kf, sizeof(float) * 6 * (size_t)H1 * H2 * H3)) != cudaSuccess) return fail(e, "malloc kfield");
  int blocks = (int)((nsym + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  DEMAG_LAUNCH(P, kFamSetup, st,
               fft3d_symbols_kernel<<<blocks, 256, 0, st>>>(P->M, P->glen, hstride, n1, n2, n3, L1, L2, L3, P->gen64,
                                                            sym, 1));
  DEMAG_LAUNCH(P, kFamSetup, st,
               fft3d_symbols_kernel<<<blocks, 256, 0, st>>>(P->M, P->glen, hstride, n1, n2, n3, L1, L2, L3, P->gend,
                                                            sym + nsym, 0));
  DEMAG_LAUNCH(P, kFamSetup, st,
               fft3d_field_kernel_kernel<<<6 * H1 * H2, 256, 0, st>>>(P->M, hstride, H1, H2, H3, P->scale, sym,
                                                                      sym + nsym, kf));
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "fft3d field kernels");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e, "fft3d field setup");
  cudaFree(sym);
  S->kfield = kf;
  return DEMAG_OK;
}

void fft3d_destroy(demag_plan* P) {
  Fft3dState* S = static_cast<Fft3dState*>(P->f3);
  if (!S) return;
  cudaFree(S->kfield);
  cudaFree(S->hfield);
  cudaFree(S->kst);
  cudaFree(S->s1);
  cudaFree(S->s2);
  delete S;
  P->f3 = nullptr;
}

// potential (field == false: one output component through P3) or stray
// field (three output components through the field P3)
static demag_status fft3d_run(demag_plan* P, const float* m, float* out, bool field, cudaStream_t st) {
  demag_status rc = field ? fft3d_prepare_field(P, st) : fft3d_prepare(P, st);
  if (rc != DEMAG_OK) return rc;
  const Fft3dState* S = static_cast<const Fft3dState*>(P->f3);
  Fft3dArgs a;
  a.nco = field ? 3 : 1;
  a.kfield = S->kfield;
  a.n1 = P->n[0];
  a.n2 = P->n[1];
  a.n3 = P->n[2];
  a.L1 = P->L[0];
  a.L2 = P->L[1];
  a.L3 = P->L[2];
  a.H1 = a.L1 / 2 + 1;
  a.H2 = a.L2 / 2 + 1;
  a.H3 = a.L3 / 2 + 1;
  a.m = m;
  a.s1 = S->s1;
  a.s2 = S->s2;
  a.phi = out;
  a.kst = S->kst;
  const int l1 = S->logL[0], l2 = S->logL[1], l3 = S->logL[2];
  const int G1 = f3_fibres(1 << l1), G2 = f3_fibres(1 << l2), G3 = f3_fibres_p3(1 << l3);
  auto cdiv = [](long x, long y) { return (int)((x + y - 1) / y); };
  a.tw = P->twid[0];
  if ((rc = dispatch_pass(P, l1, 1, a, 3 * a.n3 * cdiv(a.n2, 2 * G1), st)) != DEMAG_OK) return rc;
  a.tw = P->twid[1];
  if ((rc = dispatch_pass(P, l2, 2, a, 3 * a.H1 * cdiv(a.n3, G2), st)) != DEMAG_OK) return rc;
  a.tw = P->twid[2];
  if ((rc = dispatch_pass(P, l3, field ? 6 : 3, a, a.H1 * cdiv(a.L2, G3), st)) != DEMAG_OK) return rc;
  a.tw = P->twid[1];
  if ((rc = dispatch_pass(P, l2, 4, a, a.nco * a.n3 * cdiv(a.H1, G2), st)) != DEMAG_OK) return rc;
  a.tw = P->twid[0];
  return dispatch_pass(P, l1, 5, a, cdiv((long)a.nco * a.n2 * a.n3, 2 * G1), st);
}

demag_status fft3d_forward(demag_plan* P, const float* m, float* phi, cudaStream_t st) {
  return fft3d_run(P, m, phi, false, st);
}

// energy += -1/2 V sum_i m_i . h_i (FP64, one atomic per block), grad = -V h
__global__ void field_energy_kernel(long count, const float* m, const float* h, double half_vol, float vol,
                                    double* energy, float* grad) {
  __shared__ double red[32];
  double acc = 0.0;  // FP32 partial sums of 8 products, added in FP64
  float part = 0.f;
  int cnt = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const float hv = h[i];
    part = fmaf(m[i], hv, part);
    if (++cnt == 8) {
      acc += (double)part;
      part = 0.f;
      cnt = 0;
    }
    if (grad) grad[i] = -vol * hv;
  }
  acc += (double)part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(energy, -half_vol * t);
  }
}

demag_status fft3d_energy(demag_plan* P, const float* m, double* energy, float* grad, cudaStream_t st) {
  demag_status rc = fft3d_prepare_field(P, st);
  if (rc != DEMAG_OK) return rc;
  Fft3dState* S = static_cast<Fft3dState*>(P->f3);
  const long count = 3L * (long)field_size(P);
  if (!S->hfield) DEMAG_CUDA(P, cudaMalloc(&S->hfield, sizeof(float) * count));
  rc = fft3d_run(P, m, S->hfield, true, st);
  if (rc != DEMAG_OK) return rc;
  const double vol = P->h[0] * P->h[1] * P->h[2];
  DEMAG_CUDA(P, cudaMemsetAsync(energy, 0, sizeof(double), st));
  long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  DEMAG_LAUNCH(P, kFamEnergy, st,
               field_energy_kernel<<<(int)blocks, 256, 0, st>>>(count, m, S->hfield, 0.5 * vol, (float)vol, energy,
                                                               grad));
  DEMAG_LAUNCHED(P, "field_energy_kernel");
  return DEMAG_OK;
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_stray_field_fft(demag_plan* P, const float* m, float* hd, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_stray_field_fft: plan is NULL");
  if (!m || !hd) return set_error(P, DEMAG_EINVAL, "demag_stray_field_fft: NULL pointer");
  demag_status u = require_uniform(P, "demag_stray_field_fft");
  if (u != DEMAG_OK) return u;
  return fft3d_run(P, m, hd, true, (cudaStream_t)stream);
}

extern "C" demag_status demag_energy_field_fft(demag_plan* P, const float* m, double* energy, float* grad,
                                               void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_energy_field_fft: plan is NULL");
  if (!m || !energy) return set_error(P, DEMAG_EINVAL, "demag_energy_field_fft: NULL pointer");
  demag_status u = require_uniform(P, "demag_energy_field_fft");
  if (u != DEMAG_OK) return u;
  return fft3d_energy(P, m, energy, grad, (cudaStream_t)stream);
}

extern "C" demag_status demag_apply_full_fft(demag_plan* P, const float* m, float* phi, void* stream) {
  if (!P) return set_error(nullptr, DEMAG_EINVAL, "demag_apply_full_fft: plan is NULL");
  if (!m || !phi) return set_error(P, DEMAG_EINVAL, "demag_apply_full_fft: NULL pointer");
  return fft3d_forward(P, m, phi, (cudaStream_t)stream);
}
