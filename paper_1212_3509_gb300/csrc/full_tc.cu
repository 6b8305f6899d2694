// Full format on tcgen05 tensor cores: split-precision (BF16x3) mode products.
//
// The same chain as full_simt.cu (Cor. 3, Eq. kron_operator, as mode products
// of Eq. modemul; 8 GEMMs per node; node sum folded into the last
// contraction; transposed stores rotate the axes), with every GEMM operand x
// carried as x_hi = bf16(x), x_lo = bf16(x - x_hi) and each product formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with FP32 accumulation in tensor memory.
//
// Kernel: persistent, one CTA (192 threads) per SM, warp-specialised:
//   warp 0      TMA producer: loads A_hi, A_lo (128 x 32) and B_hi, B_lo
//               (BN x 32) k-blocks into a 4-stage shared-memory ring,
//   warp 1      MMA issuer: 2 k-steps x 3 tcgen05.mma (M = 128, N = BN,
//               K = 16) per stage into one of two TMEM accumulators
//               (2 x 256 columns),
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

constexpr int kBM = 128, kBN = 256, kBK = 32;     // k-block: 32 bf16 = one 64-byte swizzled row
constexpr int kStages = 4;
constexpr int kTileA = kBM * kBK * 2;              // 8 KB
constexpr int kTileB = kBN * kBK * 2;              // 16 KB
constexpr int kStageBytes = 2 * kTileA + 2 * kTileB;  // 48 KB
constexpr int kBarBytes = 256;
constexpr int kSmemBytes = kStages * kStageBytes + kBarBytes + 1024;
constexpr int kTcThreads = 192;
constexpr int kMaxTcJobs = 3 * kMaxTerms + 8;
constexpr int kMaxTcPairs = 4 * kMaxTerms + 8;
constexpr uint64_t kWaitNs = 2000000000ull;        // 2 s bound on every wait
constexpr uint32_t kSwizzle64 = 4;                 // descriptor code of SWIZZLE_64B
constexpr uint32_t kSBO = 8 * 64;                  // 8 rows x 64 bytes per swizzle atom

enum TcOut { kOutSplit = 0, kOutF32 = 1 };

struct TcJob {
  int pair0, npairs, out_field, pad;
};

struct TcParams {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // 3D maps: (K, rows, field | matrix)
  void* out_hi;                        // split: bf16 hi plane base; f32: float base
  void* out_lo;                        // split: bf16 lo plane base
  long long field_elems;               // elements per output field
  long long s_a;                       // output stride of the column index a
  int ldC, n_inner;                    // output row stride and row split (outer, inner)
  int rows, n_a, kblocks, bn, mode;
  float alpha;
  int njobs, m_tiles, n_tiles, total_tiles;
  int* status;
  TcJob jobs[kMaxTcJobs];
  short2 pairs[kMaxTcPairs];           // (A field, B matrix)
};

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

__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
  uint64_t* empty = full + kStages;
  uint64_t* tfull = empty + kStages;   // [2]
  uint64_t* tempty = tfull + 2;        // [2]
  uint64_t* drain = tempty + 2;        // [1]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
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
      const uint32_t bytes = 2 * kTileA + 2 * (uint32_t)p.bn * kBK * 2;
      int s = 0;
      uint32_t ph = 0;
      for (int tile = blockIdx.x; tile < p.total_tiles && !*abort; tile += gridDim.x) {
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
            ptx::tma_load_3d(st, &p.a_hi, &full[s], kb * kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + kTileA, &p.a_lo, &full[s], kb * kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + 2 * kTileA, &p.b_hi, &full[s], kb * kBK, nt * kBN, pr.y);
            ptx::tma_load_3d(st + 2 * kTileA + kTileB, &p.b_lo, &full[s], kb * kBK, nt * kBN, pr.y);
            if (++s == kStages) { s = 0; ph ^= 1; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = ptx::instr_desc(1, kBM, (uint32_t)p.bn);
      int s = 0;
      uint32_t ph = 0, tph = 0;
      int buf = 0;
      for (int tile = blockIdx.x; tile < p.total_tiles && !*abort; tile += gridDim.x) {
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
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 bf16 along K
              const uint64_t ah = ptx::smem_desc(st + off, kSBO, kSwizzle64);
              const uint64_t al = ptx::smem_desc(st + kTileA + off, kSBO, kSwizzle64);
              const uint64_t bh = ptx::smem_desc(st + 2 * kTileA + off, kSBO, kSwizzle64);
              const uint64_t bl = ptx::smem_desc(st + 2 * kTileA + kTileB + off, kSBO, kSwizzle64);
              ptx::mma_bf16(d, ah, bh, idesc, acc);
              ptx::mma_bf16(d, ah, bl, idesc, 1u);
              ptx::mma_bf16(d, al, bh, idesc, 1u);
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
    for (int tile = blockIdx.x; tile < p.total_tiles && !*abort; tile += gridDim.x) {
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
      for (int c0 = 0; c0 < p.bn; c0 += 32) {
        uint32_t r[32];
        ptx::tmem_ld32(taddr + (uint32_t)c0, r);
        ptx::tmem_ld_wait();
        if (valid) {
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const int a = nt * kBN + c0 + jj;
            if (a < p.n_a) {
              const float x = p.alpha * __uint_as_float(r[jj]);
              const long long idx = rbase + (long long)a * p.s_a;
              if (p.mode == kOutSplit) {
                const __nv_bfloat16 hi = __float2bfloat16_rn(x);
                const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
                reinterpret_cast<__nv_bfloat16*>(p.out_hi)[idx] = hi;
                reinterpret_cast<__nv_bfloat16*>(p.out_lo)[idx] = lo;
              } else {
                reinterpret_cast<float*>(p.out_hi)[idx] = x;
              }
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

// hi/lo split of a [fields][rows][n] FP32 tensor into [fields][rows][ld] BF16 planes
__global__ void split_rows_kernel(const float* __restrict__ x, long long nrows, int n, int ld,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const long long total = nrows * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / n;
    const int c = (int)(i - r * n);
    const float v = x[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const long long o = r * ld + c;
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Dense Toeplitz factors of one axis, hi/lo, [M][2][n][ld]; the third axis
// carries the scale c s omega_k.
__global__ void tc_factor_kernel(int M, int glen, int axis, int n, int ld, const double* gen, const double* scale,
                                 __nv_bfloat16* hi, __nv_bfloat16* lo) {
  const long long total = (long long)M * 2 * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(i % n);
    const long long t = i / n;
    const int ii = (int)(t % n);
    const int kt = (int)(t / n);  // k*2 + type
    double v = gen[((long long)kt * 3 + axis) * glen + (ii - jj + n - 1)];
    if (axis == 2) v *= scale[kt / 2];
    const float f = (float)v;
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    const long long o = ((long long)kt * n + ii) * ld + jj;
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(f - __bfloat162float(h));
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

// 3D BF16 map over [dim2][dim1][ld] with logical inner extent dim0 <= ld; box (32, box1, 1), 64B swizzle.
static bool make_map(CUtensorMap* m, void* base, uint64_t dim0, uint64_t dim1, uint64_t dim2, uint64_t ld,
                     uint32_t box1) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {dim0, dim1, dim2};
  cuuint64_t strides[2] = {ld * 2, ld * dim1 * 2};
  cuuint32_t box[3] = {(cuuint32_t)kBK, box1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Per-plan tensor-core state (BF16x3).
struct TcState {
  int ld[3];              // padded row lengths (multiples of 8 bf16 = 16 bytes)
  int bn[3];              // N tile width per axis
  __nv_bfloat16* B[3][2];  // per axis: hi / lo factors [M][2][n][ld]
  __nv_bfloat16* X[2];     // split input: [3][n3 n2][ld1]
  __nv_bfloat16* buf1[2];  // [3M][n1 n3][ld2]
  __nv_bfloat16* buf2[2];  // [3M][n2 n1][ld3]
  CUtensorMap mapB[3][2];
  CUtensorMap mapX[2], map1[2], map2[2];
  int* status;
  size_t bytes;
};

static TcState* state(demag_plan* P) { return reinterpret_cast<TcState*>(P->tc); }

size_t tc_workspace_bytes(const demag_plan* P, demag_precision prec) {
  (void)prec;
  size_t b = 0;
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2];
  const size_t l1 = round_up(n1, 8), l2 = round_up(n2, 8), l3 = round_up(n3, 8);
  for (int p = 0; p < 3; ++p) b += 2 * (size_t)P->M * 2 * P->n[p] * round_up(P->n[p], 8) * 2;
  b += 2 * 3 * (size_t)n3 * n2 * l1 * 2;
  b += 2 * 3 * (size_t)P->M * n1 * n3 * l2 * 2;
  b += 2 * 3 * (size_t)P->M * n2 * n1 * l3 * 2;
  return b;
}

void tc_destroy(demag_plan* P) {
  TcState* S = state(P);
  if (!S) return;
  for (int p = 0; p < 3; ++p)
    for (int h = 0; h < 2; ++h) cudaFree(S->B[p][h]);
  for (int h = 0; h < 2; ++h) {
    cudaFree(S->X[h]);
    cudaFree(S->buf1[h]);
    cudaFree(S->buf2[h]);
  }
  cudaFree(S->status);
  delete S;
  P->tc = nullptr;
}

static int grid_blocks(long long count) {
  long long b = (count + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

demag_status tc_prepare(demag_plan* P, demag_precision prec, cudaStream_t st) {
  if (prec != DEMAG_BF16X3) return set_error(P, DEMAG_EUNSUPPORTED, "tensor-core form %d is not built", (int)prec);
  if (P->tc) return DEMAG_OK;
  if (!encode_fn()) return set_error(P, DEMAG_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  TcState* S = new TcState();
  memset(S, 0, sizeof(*S));
  P->tc = S;
  for (int p = 0; p < 3; ++p) {
    S->ld[p] = round_up(P->n[p], 8);
    S->bn[p] = P->n[p] >= kBN ? kBN : round_up(P->n[p], 16);
  }
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    S->bytes += bytes;
    return cudaMemsetAsync(*ptr, 0, bytes, st) == cudaSuccess;
  };
  bool ok = true;
  for (int p = 0; p < 3 && ok; ++p)
    for (int h = 0; h < 2 && ok; ++h)
      ok = alloc((void**)&S->B[p][h], (size_t)M * 2 * P->n[p] * S->ld[p] * 2);
  for (int h = 0; h < 2 && ok; ++h) {
    ok = ok && alloc((void**)&S->X[h], 3 * (size_t)n3 * n2 * S->ld[0] * 2);
    ok = ok && alloc((void**)&S->buf1[h], 3 * (size_t)M * n1 * n3 * S->ld[1] * 2);
    ok = ok && alloc((void**)&S->buf2[h], 3 * (size_t)M * n2 * n1 * S->ld[2] * 2);
  }
  ok = ok && alloc((void**)&S->status, sizeof(int));
  if (!ok) {
    tc_destroy(P);
    return set_error(P, DEMAG_ENOMEM, "tensor-core workspace allocation failed");
  }
  for (int p = 0; p < 3; ++p) {
    long long total = (long long)M * 2 * P->n[p] * P->n[p];
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<<<grid_blocks(total), 256, 0, st>>>(M, P->glen, p, P->n[p], S->ld[p], P->gen64,
                                                                      P->scale, S->B[p][0], S->B[p][1]));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  for (int h = 0; h < 2; ++h) {
    for (int p = 0; p < 3; ++p)
      ok = ok && make_map(&S->mapB[p][h], S->B[p][h], P->n[p], P->n[p], 2 * M, S->ld[p], S->bn[p]);
    ok = ok && make_map(&S->mapX[h], S->X[h], n1, (uint64_t)n3 * n2, 3, S->ld[0], kBM);
    ok = ok && make_map(&S->map1[h], S->buf1[h], n2, (uint64_t)n1 * n3, 3 * M, S->ld[1], kBM);
    ok = ok && make_map(&S->map2[h], S->buf2[h], n3, (uint64_t)n2 * n1, 3 * M, S->ld[2], kBM);
  }
  if (!ok) {
    tc_destroy(P);
    return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  }
  static bool attr = false;
  if (!attr) {
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr = true;
  }
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

static demag_status launch_stage(demag_plan* P, const StageDesc& d, const std::vector<TcJob>& jobs,
                                 const std::vector<short2>& pairs, cudaStream_t st) {
  TcState* S = state(P);
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
  prm.kblocks = (d.K + kBK - 1) / kBK;
  prm.bn = d.bn;
  prm.mode = d.mode;
  prm.alpha = d.alpha;
  prm.njobs = (int)jobs.size();
  prm.m_tiles = (d.rows + kBM - 1) / kBM;
  prm.n_tiles = (d.n_a + kBN - 1) / kBN;
  prm.total_tiles = prm.njobs * prm.m_tiles * prm.n_tiles;
  prm.status = S->status;
  for (size_t i = 0; i < jobs.size(); ++i) prm.jobs[i] = jobs[i];
  for (size_t i = 0; i < pairs.size(); ++i) prm.pairs[i] = pairs[i];
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = prm.total_tiles < sms ? prm.total_tiles : sms;
  DEMAG_LAUNCH(P, kFamGemmTc, st, tc_gemm_kernel<<<grid, kTcThreads, kSmemBytes, st>>>(prm));
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

static demag_status split_input(demag_plan* P, const float* x, int fields, cudaStream_t st) {
  TcState* S = state(P);
  const long long nrows = (long long)fields * P->n[2] * P->n[1];
  DEMAG_LAUNCH(P, kFamSplit, st,
               split_rows_kernel<<<grid_blocks(nrows * P->n[0]), 256, 0, st>>>(x, nrows, P->n[0], S->ld[0],
                                                                                 S->X[0], S->X[1]));
  DEMAG_LAUNCHED(P, "split_rows_kernel");
  return DEMAG_OK;
}

// matrix index of (node k, type) in the per-axis factor maps
static short mat(int k, int type) { return (short)(2 * k + type); }

demag_status tc_forward(demag_plan* P, const float* m, float* phi, demag_precision prec, cudaStream_t st) {
  demag_status s = tc_prepare(P, prec, st);
  if (s != DEMAG_OK) return s;
  TcState* S = state(P);
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  s = split_input(P, m, 3, st);
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
    s = launch_stage(P, d, jobs, pairs, st);
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
    s = launch_stage(P, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 3 with the node sum: phi = sum_k U_k x_3 S E + V_k x_3 S F; rows (i2', i1') -> [i3'][i2'][i1']
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    jobs.push_back(job(0, 2 * M, 0));
    for (int k = 0; k < M; ++k) {
      pairs.push_back(make_short2((short)(2 * k), mat(k, 0)));
      pairs.push_back(make_short2((short)(2 * k + 1), mat(k, 1)));
    }
    StageDesc d{{&S->map2[0], &S->map2[1]}, {&S->mapB[2][0], &S->mapB[2][1]}, n2 * n1, n3, n3, S->bn[2],
                phi, nullptr, (long long)n3 * n2 * n1, (long long)n2 * n1, n1, n1, kOutF32, 1.f};
    s = launch_stage(P, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  return DEMAG_OK;
}

demag_status tc_adjoint(demag_plan* P, const float* y, float* g, demag_precision prec, cudaStream_t st) {
  demag_status s = tc_prepare(P, prec, st);
  if (s != DEMAG_OK) return s;
  TcState* S = state(P);
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  s = split_input(P, y, 1, st);
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
    s = launch_stage(P, d, jobs, pairs, st);
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
    s = launch_stage(P, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  // mode 3 with the node sum: g_q = -sum_k Z_kq x_3 S T_{k,q,3}
  {
    std::vector<TcJob> jobs;
    std::vector<short2> pairs;
    for (int q = 0; q < 3; ++q) {
      jobs.push_back(job((int)pairs.size(), M, q));
      for (int k = 0; k < M; ++k) pairs.push_back(make_short2((short)(3 * k + q), mat(k, q == 2 ? 1 : 0)));
    }
    StageDesc d{{&S->map2[0], &S->map2[1]}, {&S->mapB[2][0], &S->mapB[2][1]}, n2 * n1, n3, n3, S->bn[2],
                g, nullptr, (long long)n3 * n2 * n1, (long long)n2 * n1, n1, n1, kOutF32, -1.f};
    s = launch_stage(P, d, jobs, pairs, st);
    if (s != DEMAG_OK) return s;
  }
  return DEMAG_OK;
}

demag_status tc_sync_status(demag_plan* P, cudaStream_t st) {
  TcState* S = state(P);
  if (!S) return DEMAG_OK;
  int h = 0;
  DEMAG_CUDA(P, cudaMemcpyAsync(&h, S->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  DEMAG_CUDA(P, cudaStreamSynchronize(st));
  if (h) {
    DEMAG_CUDA(P, cudaMemsetAsync(S->status, 0, sizeof(int), st));
    return set_error(P, (demag_status)h, "tensor-core kernel reported status %d (a bounded wait gave up)", h);
  }
  return DEMAG_OK;
}

}  // namespace demag
