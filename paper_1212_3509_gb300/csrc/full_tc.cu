// Full format on tcgen05 tensor cores: split-precision mode products
// (BF16x3 and TF32x3).
//
// The same chain as full_simt.cu (Cor. 3, Eq. kron_operator, as mode products
// of Eq. modemul; 8 GEMMs per node; node sum folded into the last
// contraction; transposed stores rotate the axes), with every GEMM operand x
// carried as x_hi = round(x), x_lo = round(x - x_hi) in BF16 or TF32 and each
// product formed as A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation
// in tensor memory.
//
// Kernel: persistent, one CTA (192 threads) per SM, warp-specialised:
//   warp 0      TMA producer: loads A_hi, A_lo (128 rows) and B_hi, B_lo
//               (BN rows) k-blocks of 64-byte rows (32 BF16 or 16 TF32
//               elements) into a 4-stage shared-memory ring,
//   warp 1      MMA issuer: 2 k-steps x 3 tcgen05.mma (M = 128, N = BN) per
//               stage into one of two TMEM accumulators (2 x 256 columns),
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (one TMEM lane per
//               thread = one output row), then either the hi/lo split of the
//               next stage's operand or the final FP32 field, stored
//               transposed (consecutive threads write consecutive addresses).
// Tiles are (job, 128-row block, BN-column block); a job is one output field
// with a list of (A field, B matrix) pairs whose contractions it sums.
#include <cuda_bf16.h>

#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace demag {

constexpr int kBM = 128, kBN = 256;
constexpr int kRowBytes = 64;                      // one 64-byte swizzled row per k-block
constexpr int kStages = 4;
constexpr int kTileA = kBM * kRowBytes;            // 8 KB
constexpr int kTileB = kBN * kRowBytes;            // 16 KB
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;  // 48 KB
constexpr int kBarBytes = 256;
constexpr int kSmemBytes = kStages * kStageBytes + kBarBytes + 1024;
constexpr int kTcThreads = 192;
constexpr int kMaxTcJobs = 3 * kMaxTerms + 8;
constexpr int kMaxTcPairs = 4 * kMaxTerms + 8;
constexpr uint64_t kWaitNs = 2000000000ull;        // 2 s bound on every wait
constexpr uint32_t kSwizzle64 = 4;                 // descriptor code of SWIZZLE_64B
constexpr uint32_t kSBO = 8 * kRowBytes;           // 8 rows x 64 bytes per swizzle atom

enum TcOut { kOutSplit = 0, kOutF32 = 1 };

// Element traits of the two split forms.
struct Bf16Form {
  using T = __nv_bfloat16;
  static constexpr int kElem = 2;
  static constexpr int kBK = kRowBytes / kElem;    // 32 elements per k-block
  static constexpr uint32_t kFormat = 1;           // instruction-descriptor code of BF16
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    ptx::mma_bf16(d, a, b, idesc, acc);
  }
  __device__ static void split(float x, T& hi, T& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
  }
};

struct Tf32Form {
  using T = float;                                 // TF32 values in 32-bit containers
  static constexpr int kElem = 4;
  static constexpr int kBK = kRowBytes / kElem;    // 16 elements per k-block
  static constexpr uint32_t kFormat = 2;           // instruction-descriptor code of TF32
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    ptx::mma_tf32(d, a, b, idesc, acc);
  }
  __device__ static float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  __device__ static void split(float x, T& hi, T& lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - hi);
  }
};

struct TcJob {
  int pair0, npairs, out_field, pad;
};

struct TcParams {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // 3D maps: (K, rows, field | matrix)
  void* out_hi;                        // split: hi plane base; f32: float base
  void* out_lo;                        // split: lo plane base
  long long field_elems;               // elements per output field
  long long s_a;                       // output stride of the column index a
  int ldC, n_inner;                    // output row stride and row split (outer, inner)
  int rows, n_a, kblocks, bn, mode;
  float alpha;
  int njobs, m_tiles, n_tiles, total_tiles;
  int* status;
  int* tile_counter;                   // zeroed before the launch; tiles are taken in order
  TcJob jobs[kMaxTcJobs];
  short2 pairs[kMaxTcPairs];           // (A field, B matrix)
};

constexpr int kRing = 4;               // tile ids handed from the producer to the other roles

__device__ __forceinline__ void tile_coords(const TcParams& p, int tile, int& j, int& mt, int& nt) {
  // job fastest: consecutive tiles share the A row block (L2 reuse across nodes)
  j = tile % p.njobs;
  int rest = tile / p.njobs;
  nt = rest % p.n_tiles;
  mt = rest / p.n_tiles;
}

__device__ __forceinline__ void tc_fail(volatile int* abort, int* status) {
  *abort = 1;
  atomicExch(status, (int)DEMAG_ETIMEOUT);
}

template <class F>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  using T = typename F::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;   // [2]
  uint64_t* tempty = tfull + 2;        // [2]
  uint64_t* drain = tempty + 2;        // [1]
  uint64_t* sfull = drain + 1;         // [kRing] a tile id is in the ring slot
  uint64_t* sempty = sfull + kRing;    // [kRing] the MMA thread and the 4 epilogue warps read it
  volatile int* ring = reinterpret_cast<volatile int*>(sempty + kRing);  // [kRing]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sempty + kRing) + kRing;
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&tfull[b], 1);
      ptx::mbar_init(&tempty[b], 4);
    }
    for (int i = 0; i < kRing; ++i) {
      ptx::mbar_init(&sfull[i], 1);
      ptx::mbar_init(&sempty[i], 5);
    }
    ptx::mbar_init(drain, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  bool issued_mma = false;

  if (warp == 0) {
    if (lane == 0) {
      ptx::prefetch_tmap(&p.a_hi);
      ptx::prefetch_tmap(&p.a_lo);
      ptx::prefetch_tmap(&p.b_hi);
      ptx::prefetch_tmap(&p.b_lo);
      const uint32_t bytes = 2 * kTileA + 2 * (uint32_t)p.bn * kRowBytes;
      int s = 0;
      uint32_t ph = 0;
      int rs = 0;
      uint32_t rph = 0;
      while (!*abort) {
        // take the next tile and hand its id to the MMA and epilogue roles
        if (!ptx::mbar_wait(&sempty[rs], rph ^ 1, abort, kWaitNs)) {
          tc_fail(abort, p.status);
          break;
        }
        const int tile = atomicAdd(p.tile_counter, 1);
        ring[rs] = tile < p.total_tiles ? tile : -1;
        ptx::mbar_arrive(&sfull[rs]);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile >= p.total_tiles) break;
        int j, mt, nt;
        tile_coords(p, tile, j, mt, nt);
        const TcJob& J = p.jobs[j];
        for (int pi = 0; pi < J.npairs && !*abort; ++pi) {
          const short2 pr = p.pairs[J.pair0 + pi];
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!ptx::mbar_wait(&empty[s], ph ^ 1, abort, kWaitNs)) {
              tc_fail(abort, p.status);
              break;
            }
            uint8_t* st = smem + s * kStageBytes;
            ptx::mbar_arrive_expect_tx(&full[s], bytes);
            ptx::tma_load_3d(st, &p.a_hi, &full[s], kb * F::kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + kTileA, &p.a_lo, &full[s], kb * F::kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + 2 * kTileA, &p.b_hi, &full[s], kb * F::kBK, nt * kBN, pr.y);
            ptx::tma_load_3d(st + 2 * kTileA + kTileB, &p.b_lo, &full[s], kb * F::kBK, nt * kBN, pr.y);
            if (++s == kStages) { s = 0; ph ^= 1; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = ptx::instr_desc(F::kFormat, kBM, (uint32_t)p.bn);
      int s = 0;
      uint32_t ph = 0, tph = 0;
      int buf = 0;
      int rs = 0;
      uint32_t rph = 0;
      while (!*abort) {
        if (!ptx::mbar_wait(&sfull[rs], rph, abort, kWaitNs)) {
          tc_fail(abort, p.status);
          break;
        }
        const int tile = ring[rs];
        ptx::mbar_arrive(&sempty[rs]);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile < 0) break;
        int j, mt, nt;
        tile_coords(p, tile, j, mt, nt);
        const TcJob& J = p.jobs[j];
        if (!ptx::mbar_wait(&tempty[buf], tph ^ 1, abort, kWaitNs)) {
          tc_fail(abort, p.status);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(buf * kBN);
        uint32_t acc = 0;
        bool ok = true;
        for (int pi = 0; pi < J.npairs && ok; ++pi) {
          for (int kb = 0; kb < p.kblocks; ++kb) {
            if (!ptx::mbar_wait(&full[s], ph, abort, kWaitNs)) {
              tc_fail(abort, p.status);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t st = ptx::smem_u32(smem + s * kStageBytes);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint32_t off = kk * 32;  // one MMA consumes 32 bytes of K
              const uint64_t ah = ptx::smem_desc(st + off, kSBO, kSwizzle64);
              const uint64_t al = ptx::smem_desc(st + kTileA + off, kSBO, kSwizzle64);
              const uint64_t bh = ptx::smem_desc(st + 2 * kTileA + off, kSBO, kSwizzle64);
              const uint64_t bl = ptx::smem_desc(st + 2 * kTileA + kTileB + off, kSBO, kSwizzle64);
              F::mma(d, ah, bh, idesc, acc);
              F::mma(d, ah, bl, idesc, 1u);
              F::mma(d, al, bh, idesc, 1u);
              acc = 1u;
            }
            issued_mma = true;
            ptx::mma_commit(&empty[s]);
            if (++s == kStages) { s = 0; ph ^= 1; }
          }
        }
        if (!ok) break;
        ptx::mma_commit(&tfull[buf]);
        buf ^= 1;
        if (buf == 0) tph ^= 1;
      }
    }
  } else {
    const int quad = warp & 3;  // TMEM lane quadrant this warp may access
    const int rloc = quad * 32 + lane;
    int buf = 0;
    uint32_t tph = 0;
    int rs = 0;
    uint32_t rph = 0;
    while (!*abort) {
      if (!ptx::mbar_wait(&sfull[rs], rph, abort, kWaitNs)) {
        tc_fail(abort, p.status);
        break;
      }
      const int tile = ring[rs];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (tile < 0) break;
      int j, mt, nt;
      tile_coords(p, tile, j, mt, nt);
      const TcJob& J = p.jobs[j];
      if (!ptx::mbar_wait(&tfull[buf], tph, abort, kWaitNs)) {
        tc_fail(abort, p.status);
        break;
      }
      ptx::tc_fence_after();
      const int row = mt * kBM + rloc;
      const bool valid = row < p.rows;
      const int outer = row / p.n_inner, inner = row - outer * p.n_inner;
      const long long rbase = (long long)J.out_field * p.field_elems + (long long)outer * p.ldC + inner;
      const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * kBN);
      const int a0 = nt * kBN;
      const int acount = min(p.bn, p.n_a - a0);  // columns of this tile that exist
      for (int c0 = 0; c0 < p.bn; c0 += 32) {
        uint32_t r[32];
        ptx::tmem_ld32(taddr + (uint32_t)c0, r);
        ptx::tmem_ld_wait();
        if (valid) {
          if (p.mode == kOutSplit) {
            T* hp = reinterpret_cast<T*>(p.out_hi) + rbase + (long long)(a0 + c0) * p.s_a;
            T* lp = reinterpret_cast<T*>(p.out_lo) + rbase + (long long)(a0 + c0) * p.s_a;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              if (c0 + jj < acount) {
                T hi, lo;
                F::split(__uint_as_float(r[jj]), hi, lo);
                *hp = hi;
                *lp = lo;
              }
              hp += p.s_a;
              lp += p.s_a;
            }
          } else {
            float* op = reinterpret_cast<float*>(p.out_hi) + rbase + (long long)(a0 + c0) * p.s_a;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              if (c0 + jj < acount) *op = p.alpha * __uint_as_float(r[jj]);
              op += p.s_a;
            }
          }
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[buf]);
      buf ^= 1;
      if (buf == 0) tph ^= 1;
    }
  }

  // teardown: after an abort let in-flight MMAs and copies land (bounded)
  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (*abort) {
    if (warp == 1 && lane == 0 && issued_mma) {
      volatile int no_abort = 0;
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, &no_abort, kWaitNs);
    }
    if (threadIdx.x == 0) {
      const uint64_t t0 = ptx::globaltimer();
      while (ptx::globaltimer() - t0 < 1000000ull) {
      }
    }
    __syncthreads();
  }
  if (warp == 1) ptx::tmem_dealloc(tmem_base, 512);
}

// ---------------------------------------------------------------- operand preparation

// hi/lo split of a [fields][rows][n] FP32 tensor into [fields][rows][ld] planes
template <class F>
__global__ void split_rows_kernel(const float* __restrict__ x, long long nrows, int n, int ld,
                                  typename F::T* __restrict__ hi, typename F::T* __restrict__ lo) {
  const long long total = nrows * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / n;
    const int c = (int)(i - r * n);
    typename F::T h, l;
    F::split(x[i], h, l);
    const long long o = r * ld + c;
    hi[o] = h;
    lo[o] = l;
  }
}

// Dense Toeplitz factors of one axis, hi/lo, [M][2][n][ld]; the third axis
// carries the scale c s omega_k.
template <class F>
__global__ void tc_factor_kernel(int M, int glen, int axis, int n, int ld, const double* gen, const double* scale,
                                 typename F::T* hi, typename F::T* lo) {
  const long long total = (long long)M * 2 * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(i % n);
    const long long t = i / n;
    const int ii = (int)(t % n);
    const int kt = (int)(t / n);  // k*2 + type
    double v = gen[((long long)kt * 3 + axis) * glen + (ii - jj + n - 1)];
    if (axis == 2) v *= scale[kt / 2];
    typename F::T h, l;
    F::split((float)v, h, l);
    const long long o = ((long long)kt * n + ii) * ld + jj;
    hi[o] = h;
    lo[o] = l;
  }
}

// ---------------------------------------------------------------- host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3D map over [dim2][dim1][ld] with logical inner extent dim0 <= ld; box (64 bytes, box1, 1), 64B swizzle.
static bool make_map(CUtensorMap* m, void* base, int elem_bytes, uint64_t dim0, uint64_t dim1, uint64_t dim2,
                     uint64_t ld, uint32_t box1) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {dim0, dim1, dim2};
  cuuint64_t strides[2] = {ld * elem_bytes, ld * dim1 * elem_bytes};
  cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / elem_bytes), box1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Per-plan, per-form tensor-core state.
struct TcState {
  int elem;               // bytes per element (2 BF16, 4 TF32)
  int ld[3];              // padded row lengths (16-byte multiples)
  int bn[3];              // N tile width per axis
  void* B[3][2];          // per axis: hi / lo factors [M][2][n][ld]
  void* X[2];             // split input: [3][n3 n2][ld1]
  void* buf1[2];          // [3M][n1 n3][ld2]
  void* buf2[2];          // [3M][n2 n1][ld3]
  CUtensorMap mapB[3][2];
  CUtensorMap mapX[2], map1[2], map2[2];
  int* status;
  int* counter;           // dynamic tile counter of the running launch
  float* part;            // split node-sum partial fields
  int pp3;                // (A, B) pairs per accumulator in the node-sum stage
  size_t bytes;
};

// The tensor cores accumulate into TMEM with FP32 additions that do not round
// to nearest, so the error of a long contraction grows with the number of
// MMAs accumulated into one accumulator.  The node-sum stage (2M pairs of
// length n3) is therefore split into groups of at most ~400 accumulations,
// whose FP32 partial fields are summed on CUDA cores in FP64.
static int pairs_per_split(int kblocks) {
  const int per_pair = kblocks * 6;  // 2 k-steps x 3 products per k-block
  const int pp = 400 / (per_pair > 0 ? per_pair : 1);
  return pp < 1 ? 1 : pp;
}

// out[q][i] = alpha * sum_g part[q*groups + g][i], accumulated in FP64
__global__ void reduce_parts_kernel(const float* __restrict__ part, int groups, long long N, int nout, float alpha,
                                    float* __restrict__ out) {
  const long long total = (long long)nout * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long q = idx / N, i = idx - q * N;
    const float* src = part + q * groups * N + i;
    double acc = 0.0;
    for (int g = 0; g < groups; ++g) acc += (double)src[g * N];
    out[idx] = (float)(alpha * acc);
  }
}

struct TcHolder {
  TcState* s[2] = {nullptr, nullptr};  // [0] BF16x3, [1] TF32x3
};

static int form_index(demag_precision prec) { return prec == DEMAG_TF32X3 ? 1 : 0; }

static TcState* state(demag_plan* P, demag_precision prec) {
  TcHolder* H = reinterpret_cast<TcHolder*>(P->tc);
  return H ? H->s[form_index(prec)] : nullptr;
}

size_t tc_workspace_bytes(const demag_plan* P, demag_precision prec) {
  const size_t e = prec == DEMAG_TF32X3 ? 4 : 2;
  const int al = (int)(16 / e);
  size_t b = 0;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const size_t l1 = round_up(n1, al), l2 = round_up(n2, al), l3 = round_up(n3, al);
  for (int p = 0; p < 3; ++p) b += 2 * (size_t)P->M * 2 * P->n[p] * round_up(P->n[p], al) * e;
  b += 2 * 3 * (size_t)n3 * n2 * l1 * e;
  b += 2 * 3 * (size_t)P->M * n1 * n3 * l2 * e;
  b += 2 * 3 * (size_t)P->M * n2 * n1 * l3 * e;
  return b;
}

static void free_state(TcState* S) {
  if (!S) return;
  for (int p = 0; p < 3; ++p)
    for (int h = 0; h < 2; ++h) cudaFree(S->B[p][h]);
  for (int h = 0; h < 2; ++h) {
    cudaFree(S->X[h]);
    cudaFree(S->buf1[h]);
    cudaFree(S->buf2[h]);
  }
  cudaFree(S->status);
  cudaFree(S->counter);
  cudaFree(S->part);
  delete S;
}

void tc_destroy(demag_plan* P) {
  TcHolder* H = reinterpret_cast<TcHolder*>(P->tc);
  if (!H) return;
  for (auto*& s : H->s) {
    free_state(s);
    s = nullptr;
  }
  delete H;
  P->tc = nullptr;
}

static int grid_blocks(long long count) {
  long long b = (count + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

template <class F>
static demag_status prepare_form(demag_plan* P, TcState* S, cudaStream_t st) {
  const int M = P->M;
  for (int p = 0; p < 3; ++p) {
    long long total = (long long)M * 2 * P->n[p] * P->n[p];
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<F><<<grid_blocks(total), 256, 0, st>>>(
                     M, P->glen, p, P->n[p], S->ld[p], P->gen64, P->scale, (typename F::T*)S->B[p][0],
                     (typename F::T*)S->B[p][1]));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  static bool attr = false;
  if (!attr) {
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_gemm_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr = true;
  }
  return DEMAG_OK;
}

demag_status tc_prepare(demag_plan* P, demag_precision prec, cudaStream_t st) {
  if (prec != DEMAG_BF16X3 && prec != DEMAG_TF32X3)
    return set_error(P, DEMAG_EUNSUPPORTED, "tensor-core form %d is not built", (int)prec);
  if (state(P, prec)) return DEMAG_OK;
  if (!encode_fn()) return set_error(P, DEMAG_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if (!P->tc) P->tc = new TcHolder();
  TcHolder* H = reinterpret_cast<TcHolder*>(P->tc);
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  TcState* S = new TcState();
  memset(S, 0, sizeof(*S));
  S->elem = prec == DEMAG_TF32X3 ? 4 : 2;
  const int al = 16 / S->elem;
  for (int p = 0; p < 3; ++p) {
    S->ld[p] = round_up(P->n[p], al);
    S->bn[p] = P->n[p] >= kBN ? kBN : round_up(P->n[p], 16);
  }
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    S->bytes += bytes;
    return cudaMemsetAsync(*ptr, 0, bytes, st) == cudaSuccess;
  };
  const size_t e = S->elem;
  bool ok = true;
  for (int p = 0; p < 3 && ok; ++p)
    for (int h = 0; h < 2 && ok; ++h) ok = alloc(&S->B[p][h], (size_t)M * 2 * P->n[p] * S->ld[p] * e);
  for (int h = 0; h < 2 && ok; ++h) {
    ok = ok && alloc(&S->X[h], 3 * (size_t)n3 * n2 * S->ld[0] * e);
    ok = ok && alloc(&S->buf1[h], 3 * (size_t)M * n1 * n3 * S->ld[1] * e);
    ok = ok && alloc(&S->buf2[h], 3 * (size_t)M * n2 * n1 * S->ld[2] * e);
  }
  ok = ok && alloc((void**)&S->status, sizeof(int));
  ok = ok && alloc((void**)&S->counter, sizeof(int));
  {
    const int kb3 = (n3 + kRowBytes / S->elem - 1) / (kRowBytes / S->elem);
    S->pp3 = pairs_per_split(kb3);
    const int gf = (2 * M + S->pp3 - 1) / S->pp3;   // forward: 2M pairs in one sum
    const int ga = (M + S->pp3 - 1) / S->pp3;       // adjoint: M pairs per component
    const int fields = gf > 3 * ga ? gf : 3 * ga;
    ok = ok && alloc((void**)&S->part, sizeof(float) * (size_t)fields * n1 * n2 * n3);
  }
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ENOMEM, "tensor-core workspace allocation failed");
  }
  for (int h = 0; h < 2; ++h) {
    for (int p = 0; p < 3; ++p)
      ok = ok && make_map(&S->mapB[p][h], S->B[p][h], S->elem, P->n[p], P->n[p], 2 * M, S->ld[p], S->bn[p]);
    ok = ok && make_map(&S->mapX[h], S->X[h], S->elem, n1, (uint64_t)n3 * n2, 3, S->ld[0], kBM);
    ok = ok && make_map(&S->map1[h], S->buf1[h], S->elem, n2, (uint64_t)n1 * n3, 3 * M, S->ld[1], kBM);
    ok = ok && make_map(&S->map2[h], S->buf2[h], S->elem, n3, (uint64_t)n2 * n1, 3 * M, S->ld[2], kBM);
  }
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  }
  demag_status s = prec == DEMAG_TF32X3 ? prepare_form<Tf32Form>(P, S, st) : prepare_form<Bf16Form>(P, S, st);
  if (s != DEMAG_OK) {
    free_state(S);
    return s;
  }
  H->s[form_index(prec)] = S;
  return DEMAG_OK;
}

// One GEMM stage: C = alpha * sum over the job's pairs of A[field] * B[matrix]^T.
struct StageDesc {
  const CUtensorMap* a[2];
  const CUtensorMap* b[2];
  int rows, n_a, K, bn;
  void* out_hi;
  void* out_lo;
  long long field_elems, s_a;
  int ldC, n_inner, mode;
  float alpha;
};

template <class F>
static demag_status launch_stage(demag_plan* P, TcState* S, const StageDesc& d, const std::vector<TcJob>& jobs,
                                 const std::vector<short2>& pairs, cudaStream_t st) {
  thread_local static TcParams prm;  // host staging; the launch copies the parameters at enqueue
  if ((int)jobs.size() > kMaxTcJobs || (int)pairs.size() > kMaxTcPairs)
    return set_error(P, DEMAG_EUNSUPPORTED, "too many GEMM jobs for one launch");
  prm.a_hi = *d.a[0];
  prm.a_lo = *d.a[1];
  prm.b_hi = *d.b[0];
  prm.b_lo = *d.b[1];
  prm.out_hi = d.out_hi;
  prm.out_lo = d.out_lo;
  prm.field_elems = d.field_elems;
  prm.s_a = d.s_a;
  prm.ldC = d.ldC;
  prm.n_inner = d.n_inner;
  prm.rows = d.rows;
  prm.n_a = d.n_a;
  prm.kblocks = (d.K + F::kBK - 1) / F::kBK;
  prm.bn = d.bn;
  prm.mode = d.mode;
  prm.alpha = d.alpha;
  prm.njobs = (int)jobs.size();
  prm.m_tiles = (d.rows + kBM - 1) / kBM;
  prm.n_tiles = (d.n_a + kBN - 1) / kBN;
  prm.total_tiles = prm.njobs * prm.m_tiles * prm.n_tiles;
  prm.status = S->status;
  prm.tile_counter = S->counter;
  for (size_t i = 0; i < jobs.size(); ++i) prm.jobs[i] = jobs[i];
  for (size_t i = 0; i < pairs.size(); ++i) prm.pairs[i] = pairs[i];
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = prm.total_tiles < sms ? prm.total_tiles : sms;
  DEMAG_CUDA(P, cudaMemsetAsync(S->counter, 0, sizeof(int), st));
  DEMAG_LAUNCH(P, kFamGemmTc, st, tc_gemm_kernel<F><<<grid, kTcThreads, kSmemBytes, st>>>(prm));
  DEMAG_LAUNCHED(P, "tc_gemm_kernel");
  return DEMAG_OK;
}

static TcJob job(int pair0, int npairs, int out_field) {
  TcJob j;
  j.pair0 = pair0;
  j.npairs = npairs;
  j.out_field = out_field;
  j.pad = 0;
  return j;
}

template <class F>
static demag_status split_input(demag_plan* P, TcState* S, const float* x, int fields, cudaStream_t st) {
  const long long nrows = (long long)fields * P->n[2] * P->n[1];
  DEMAG_LAUNCH(P, kFamSplit, st,
               split_rows_kernel<F><<<grid_blocks(nrows * P->n[0]), 256, 0, st>>>(
                   x, nrows, P->n[0], S->ld[0], (typename F::T*)S->X[0], (typename F::T*)S->X[1]));
  DEMAG_LAUNCHED(P, "split_rows_kernel");
  return DEMAG_OK;
}

// matrix index of (node k, type) in the per-axis factor maps
static short mat(int k, int type) { return (short)(2 * k + type); }

template <class F>
static demag_status forward_chain(demag_plan* P, TcState* S, const float* m, float* phi, cudaStream_t st) {
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  demag_status s = split_input<F>(P, S, m, 3, st);
  if (s != DEMAG_OK) return s;
  // mode 1: Y[k][q] = m_q x_1 T_{k,q,1}; rows (i3, i2), contraction i1 -> Y [i1'][i3][i2]
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int q = 0; q < 3; ++q)
      for (int k = 0; k < M; ++k) {
        jobs.push_back(job((int)pairs.size(), 1, 3 * k + q));
        pairs.push_back(make_short2((short)q, mat(k, q == 0 ? 1 : 0)));
      }
    StageDesc d{{&S->mapX[0], &S->mapX[1]}, {&S->mapB[0][0], &S->mapB[0][1]}, n3 * n2, n1, n1, S->bn[0],
                S->buf1[0], S->buf1[1], (long long)n1 * n3 * S->ld[1], (long long)n3 * S->ld[1], S->ld[1], n2,
                kOutSplit, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 2: U_k = Y_k1 x_2 E + Y_k2 x_2 F, V_k = Y_k3 x_2 E; rows (i1', i3) -> [i2'][i1'][i3]
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int k = 0; k < M; ++k) {
      jobs.push_back(job((int)pairs.size(), 2, 2 * k));
      pairs.push_back(make_short2((short)(3 * k + 0), mat(k, 0)));
      pairs.push_back(make_short2((short)(3 * k + 1), mat(k, 1)));
      jobs.push_back(job((int)pairs.size(), 1, 2 * k + 1));
      pairs.push_back(make_short2((short)(3 * k + 2), mat(k, 0)));
    }
    StageDesc d{{&S->map1[0], &S->map1[1]}, {&S->mapB[1][0], &S->mapB[1][1]}, n1 * n3, n2, n2, S->bn[1],
                S->buf2[0], S->buf2[1], (long long)n2 * n1 * S->ld[2], (long long)n1 * S->ld[2], S->ld[2], n3,
                kOutSplit, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 3 with the node sum: phi = sum_k U_k x_3 S E + V_k x_3 S F; rows (i2', i1') -> [i3'][i2'][i1']
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int k = 0; k < M; ++k) {
      pairs.push_back(make_short2((short)(2 * k), mat(k, 0)));
      pairs.push_back(make_short2((short)(2 * k + 1), mat(k, 1)));
    }
    const int groups = (2 * M + S->pp3 - 1) / S->pp3;
    for (int g = 0; g < groups; ++g) {
      const int p0 = g * S->pp3;
      jobs.push_back(job(p0, (2 * M - p0) < S->pp3 ? (2 * M - p0) : S->pp3, g));
    }
    const long long N = (long long)n3 * n2 * n1;
    StageDesc d{{&S->map2[0], &S->map2[1]}, {&S->mapB[2][0], &S->mapB[2][1]}, n2 * n1, n3, n3, S->bn[2],
                S->part, nullptr, N, (long long)n2 * n1, n1, n1, kOutF32, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
    DEMAG_LAUNCH(P, kFamMisc, st, reduce_parts_kernel<<<grid_blocks(N), 256, 0, st>>>(S->part, groups, N, 1, 1.f, phi));
    DEMAG_LAUNCHED(P, "reduce_parts_kernel");
  }
  return DEMAG_OK;
}

template <class F>
static demag_status adjoint_chain(demag_plan* P, TcState* S, const float* y, float* g, cudaStream_t st) {
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  demag_status s = split_input<F>(P, S, y, 1, st);
  if (s != DEMAG_OK) return s;
  // mode 1: Ya_k = y x_1 F, Yb_k = y x_1 E  (fields 2k, 2k+1 of buf1)
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int k = 0; k < M; ++k)
      for (int t = 0; t < 2; ++t) {
        jobs.push_back(job((int)pairs.size(), 1, 2 * k + t));
        pairs.push_back(make_short2((short)0, mat(k, t == 0 ? 1 : 0)));
      }
    StageDesc d{{&S->mapX[0], &S->mapX[1]}, {&S->mapB[0][0], &S->mapB[0][1]}, n3 * n2, n1, n1, S->bn[0],
                S->buf1[0], S->buf1[1], (long long)n1 * n3 * S->ld[1], (long long)n3 * S->ld[1], S->ld[1], n2,
                kOutSplit, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 2: Za = Ya x_2 E (g1), Zb = Yb x_2 F (g2), Zc = Yb x_2 E (g3)  (fields 3k+q of buf2)
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int k = 0; k < M; ++k) {
      const short src[3] = {(short)(2 * k), (short)(2 * k + 1), (short)(2 * k + 1)};
      const int typ[3] = {0, 1, 0};
      for (int q = 0; q < 3; ++q) {
        jobs.push_back(job((int)pairs.size(), 1, 3 * k + q));
        pairs.push_back(make_short2(src[q], mat(k, typ[q])));
      }
    }
    StageDesc d{{&S->map1[0], &S->map1[1]}, {&S->mapB[1][0], &S->mapB[1][1]}, n1 * n3, n2, n2, S->bn[1],
                S->buf2[0], S->buf2[1], (long long)n2 * n1 * S->ld[2], (long long)n1 * S->ld[2], S->ld[2], n3,
                kOutSplit, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 3 with the node sum: g_q = -sum_k Z_kq x_3 S T_{k,q,3}
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    const int groups = (M + S->pp3 - 1) / S->pp3;
    for (int q = 0; q < 3; ++q) {
      const int base = (int)pairs.size();
      for (int k = 0; k < M; ++k) pairs.push_back(make_short2((short)(3 * k + q), mat(k, q == 2 ? 1 : 0)));
      for (int gi = 0; gi < groups; ++gi) {
        const int p0 = gi * S->pp3;
        jobs.push_back(job(base + p0, (M - p0) < S->pp3 ? (M - p0) : S->pp3, q * groups + gi));
      }
    }
    const long long N = (long long)n3 * n2 * n1;
    StageDesc d{{&S->map2[0], &S->map2[1]}, {&S->mapB[2][0], &S->mapB[2][1]}, n2 * n1, n3, n3, S->bn[2],
                S->part, nullptr, N, (long long)n2 * n1, n1, n1, kOutF32, 1.f};
    s = launch_stage<F>(P, S, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
    DEMAG_LAUNCH(P, kFamMisc, st,
                 reduce_parts_kernel<<<grid_blocks(3 * N), 256, 0, st>>>(S->part, groups, N, 3, -1.f, g));
    DEMAG_LAUNCHED(P, "reduce_parts_kernel");
  }
  return DEMAG_OK;
}

demag_status tc_forward(demag_plan* P, const float* m, float* phi, demag_precision prec, cudaStream_t st) {
  demag_status s = tc_prepare(P, prec, st);
  if (s != DEMAG_OK) return s;
  TcState* S = state(P, prec);
  return prec == DEMAG_TF32X3 ? forward_chain<Tf32Form>(P, S, m, phi, st) : forward_chain<Bf16Form>(P, S, m, phi, st);
}

demag_status tc_adjoint(demag_plan* P, const float* y, float* g, demag_precision prec, cudaStream_t st) {
  demag_status s = tc_prepare(P, prec, st);
  if (s != DEMAG_OK) return s;
  TcState* S = state(P, prec);
  return prec == DEMAG_TF32X3 ? adjoint_chain<Tf32Form>(P, S, y, g, st) : adjoint_chain<Bf16Form>(P, S, y, g, st);
}

demag_status tc_sync_status(demag_plan* P, cudaStream_t st) {
  TcHolder* H = reinterpret_cast<TcHolder*>(P->tc);
  if (!H) return DEMAG_OK;
  for (TcState* S : H->s) {
    if (!S) continue;
    int h = 0;
    DEMAG_CUDA(P, cudaMemcpyAsync(&h, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(P, cudaStreamSynchronize(st));
    if (h) {
      DEMAG_CUDA(P, cudaMemsetAsync(S->status, 0, sizeof(int), st));
      return set_error(P, (demag_status)h, "tensor-core kernel reported status %d (a bounded wait gave up)", h);
    }
  }
  return DEMAG_OK;
}

bool tc_ready(const demag_plan* P, demag_precision prec) { return state(const_cast<demag_plan*>(P), prec) != nullptr; }

}  // namespace demag
