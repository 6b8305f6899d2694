// Shared-memory Stockham FFT building blocks (power-of-two lengths).
//
// The structured formats apply each 1D Toeplitz factor through a circulant
// embedding and the convolution theorem (Sec. 4.1: DFT / IDFT definitions,
// Eq. dft and Eq. idft with omega = exp(-2 pi i k j / n); Lemmas 4-5: the DFT
// of a CP / Tucker tensor is the 1D DFT of its factor columns).  A real signal
// of length L is transformed as a complex signal of length N = L/2 (even
// samples in the real part, odd samples in the imaginary part) followed by
// the usual split step.
//
// Complex FFT: self-sorting (Stockham) mixed-radix passes.  Pass with radix R
// over sub-transforms of size Ns: item j < N/R loads x[j + r N/R] (r < R),
// multiplies by W^(r (j mod Ns) N/(Ns R)), does an R-point DFT in registers and
// stores to y[(j / Ns) Ns R + (j mod Ns) + r Ns].  Radix 16 passes first,
// then one pass of radix 2, 4 or 8 for the remaining bits.  A pass is done
// in place: all items are read into registers, the group synchronises, then
// writes.
#pragma once

#include <cuda_runtime.h>

namespace demag {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// FP32 complex add / subtract as one packed instruction on the (re, im) pair
// (add.rn.f32x2 / sub.rn.f32x2): per component the same correctly rounded
// result as a scalar add, half the issue slots of the FFT butterflies.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long ra, rb, rc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rc));
  return r;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long ra, rb, rc;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rc) : "l"(ra), "l"(rb));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rc));
  return r;
}

// exp(-2 pi i j / 16) for j = 0..15 (cos, -sin), exact zeros and ones.
__device__ __forceinline__ constexpr double w16_re(int j) {
  return j == 0 ? 1.0 : j == 1 ? 0.92387953251128675613 : j == 2 ? 0.70710678118654752440
       : j == 3 ? 0.38268343236508977173 : j == 4 ? 0.0 : j == 5 ? -0.38268343236508977173
       : j == 6 ? -0.70710678118654752440 : j == 7 ? -0.92387953251128675613 : j == 8 ? -1.0
       : j == 9 ? -0.92387953251128675613 : j == 10 ? -0.70710678118654752440
       : j == 11 ? -0.38268343236508977173 : j == 12 ? 0.0 : j == 13 ? 0.38268343236508977173
       : j == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__device__ __forceinline__ constexpr double w16_im(int j) {
  // -sin(2 pi j / 16) = cos(2 pi (j + 4) / 16)
  return w16_re((j + 4) & 15);
}

// Multiply by exp(s 2 pi i k / R) with compile-time k, R (R <= 16); s = -1
// forward, +1 inverse.  Trivial rotations compile to swaps / negations.
template <int R, int K, bool INV, typename C>
__device__ __forceinline__ C rot(C v) {
  using T = decltype(v.x);
  constexpr int j = (K * (16 / R)) & 15;
  if constexpr (j == 0) {
    return v;
  } else if constexpr (j == 4) {  // forward: -i, inverse: +i
    C r;
    if (INV) { r.x = -v.y; r.y = v.x; } else { r.x = v.y; r.y = -v.x; }
    return r;
  } else if constexpr (j == 8) {
    C r; r.x = -v.x; r.y = -v.y; return r;
  } else if constexpr (j == 12) {
    C r;
    if (INV) { r.x = v.y; r.y = -v.x; } else { r.x = -v.y; r.y = v.x; }
    return r;
  } else {
    C w;
    w.x = (T)w16_re(j);
    w.y = INV ? -(T)w16_im(j) : (T)w16_im(j);
    return cmul(v, w);
  }
}

template <int R, bool INV, int K, typename C>
__device__ __forceinline__ void dft_combine(C (&v)[R], C (&e)[R / 2], C (&o)[R / 2]) {
  if constexpr (K < R / 2) {
    C t = rot<R, K, INV>(o[K]);
    constexpr int j = (K * (16 / R)) & 15;
    if constexpr (j == 4 || j == 12) {
      // +-i: the swap and sign fold into scalar adds (a packed add would need
      // the swapped pair built first)
      v[K].x = e[K].x + t.x;
      v[K].y = e[K].y + t.y;
      v[K + R / 2].x = e[K].x - t.x;
      v[K + R / 2].y = e[K].y - t.y;
    } else {
      v[K] = cadd(e[K], t);
      v[K + R / 2] = csub(e[K], t);
    }
    dft_combine<R, INV, K + 1>(v, e, o);
  }
}

// In-register R-point DFT, radix-2 decimation in time, natural order output.
template <int R, bool INV, typename C>
__device__ __forceinline__ void dft_reg(C (&v)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else {
    C e[R / 2], o[R / 2];
#pragma unroll
    for (int i = 0; i < R / 2; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft_reg<R / 2, INV>(e);
    dft_reg<R / 2, INV>(o);
    dft_combine<R, INV, 0>(v, e, o);
  }
}

// Radix plan for N = 2^LOGN: number of radix-16 passes and the remainder radix.
template <int LOGN> struct RadixPlan {
  static constexpr int n16 = LOGN / 4;
  static constexpr int rem = 1 << (LOGN % 4);  // 1, 2, 4 or 8
  static constexpr int passes = n16 + (rem > 1 ? 1 : 0);
};

// One Stockham pass of radix R on buf[0..N) by TG threads (local id lt).
// tw(m) returns exp(-2 pi i m / N) (forward twiddle), m < N.
template <int R, int N, int TG, bool INV, typename C, typename TW>
__device__ __forceinline__ void stockham_pass(C* buf, int Ns, int lt, const TW& tw) {
  constexpr int items = N / R;
  constexpr int ipt = (items + TG - 1) / TG;
  C v[ipt][R];
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
      const int tstep = k * (N / (Ns * R));
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = buf[j + r * items];
        if (r > 0 && Ns > 1) {
          C w = tw(r * tstep);
          if (INV) w.y = -w.y;
          x = cmul(x, w);
        }
        v[it][r] = x;
      }
      dft_reg<R, INV>(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < ipt; ++it) {
    const int j = lt + it * TG;
    if (items % TG == 0 || j < items) {
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[it][r];
    }
  }
  __syncthreads();
}

// Padded shared-memory index: one spare slot per 16, so that strided
// accesses of a Stockham pass fall into distinct banks.
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
// pad16(i + r * S) = pad16(i) + r * (S + S / 16) when S is a multiple of 16
template <int S> struct PadStride { static constexpr int value = S + S / 16; };

// pw[r] = w^r for r < R by a product tree of depth <= 4 (w^2, w^4, w^8 by
// squaring, the rest as one product of those), so each power carries only a
// few roundings of the table value w.
template <int R>
__device__ __forceinline__ void powers(float2 w, float2 (&pw)[R]) {
  pw[0] = make_float2(1.f, 0.f);
  if constexpr (R > 1) pw[1] = w;
  if constexpr (R > 2) pw[2] = cmul(w, w);
  if constexpr (R > 3) pw[3] = cmul(pw[2], w);
  if constexpr (R > 4) {
    pw[4] = cmul(pw[2], pw[2]);
    pw[5] = cmul(pw[4], w);
    pw[6] = cmul(pw[4], pw[2]);
    pw[7] = cmul(pw[4], pw[3]);
  }
  if constexpr (R > 8) {
    pw[8] = cmul(pw[4], pw[4]);
#pragma unroll
    for (int r = 9; r < R; ++r) pw[r] = cmul(pw[8], pw[r - 8]);
  }
}

// Full complex FFT of length N = 2^LOGN in place on buf (unnormalised).
// All threads of the block must call it (it synchronises the block); threads
// of a group share buf.  `lt` is the thread index inside its group of TG.
template <int LOGN, int TG, bool INV, typename C, typename TW>
__device__ __forceinline__ void fft_inplace(C* buf, int lt, const TW& tw) {
  constexpr int N = 1 << LOGN;
  using P = RadixPlan<LOGN>;
  int Ns = 1;
  if constexpr (P::rem > 1) {
    stockham_pass<P::rem, N, TG, INV>(buf, Ns, lt, tw);
    Ns *= P::rem;
  }
  if constexpr (P::n16 > 0) {
#pragma unroll
    for (int p = 0; p < P::n16; ++p) {
      stockham_pass<16, N, TG, INV>(buf, Ns, lt, tw);
      Ns *= 16;
    }
  }
}

}  // namespace demag
