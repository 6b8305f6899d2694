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
//   warp 0      TMA producer: takes tiles from an atomic counter, hands their
//               ids to the other roles through a shared ring, and loads
//               A_hi, A_lo (128 rows) and B_hi, B_lo (BN rows) k-blocks of
//               64-byte rows (32 BF16 or 16 TF32 elements) into a 4-stage
//               shared-memory ring,
//   warp 1      MMA issuer: 2 k-steps x 3 tcgen05.mma (M = 128, N = BN) per
//               stage into one of two TMEM accumulators (2 x 256 columns),
//   warps 2..5  epilogue: tcgen05.ld of the accumulator (one TMEM lane per
//               thread = one output row), then the hi/lo split of the next
//               stage's operand or an FP32 field, stored transposed, through
//               shared memory and TMA bulk stores where a warp's 32 rows share
//               one outer index, else directly (consecutive threads write
//               consecutive addresses).
// A launch runs one or several "groups": a group is one GEMM stage of one
// grid (tensor maps, shapes, a job table and a pair table in device memory,
// built once per plan).  A tile is (group, job, 128-row block, BN-column
// block); a job is one output field with a list of (A field, B matrix) pairs
// whose contractions it sums.  Several grids of different shapes therefore run
// a stage in one persistent launch.
#include <cuda_bf16.h>

#include <algorithm>
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
// Epilogue warps: kEpiWarps / 4 warps share each TMEM lane quadrant and take
// its 32-column chunks in turn.  Four (one per quadrant) measured as fast as
// eight: the stage time is set by the output write traffic, not by epilogue
// latency.
#ifndef DEMAG_TC_EPI_WARPS
#define DEMAG_TC_EPI_WARPS 4
#endif
constexpr int kEpiWarps = DEMAG_TC_EPI_WARPS;
static_assert(kEpiWarps == 4 || kEpiWarps == 8, "4 or 8 epilogue warps");
constexpr int kEpiSlices = kEpiWarps / 4;          // warps per TMEM lane quadrant
constexpr int kOutBuf = 4096;                      // one 32 x 32 output chunk (2 BF16 planes or 1 FP32)
constexpr int kOutStaging = 8 * kOutBuf;           // staging buffers shared out among the epilogue warps
constexpr int kOutBufsPerWarp = kOutStaging / (kOutBuf * kEpiWarps);
constexpr int kSmemBytes = kStages * kStageBytes + kOutStaging + kBarBytes + 1024;
constexpr int kTcThreads = 64 + 32 * kEpiWarps;
constexpr int kRing = 4;                           // tile ids handed from the producer to the other roles
#ifndef DEMAG_TC_ROW_GROUP
#define DEMAG_TC_ROW_GROUP 1
#endif
constexpr int kRowGroup = DEMAG_TC_ROW_GROUP;      // default row blocks per super-block of the tile order
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
  // four consecutive values to an 8-byte aligned address
  __device__ static void store4(T* p, const T (&v)[4]) {
    uint2 u;
    u.x = (uint32_t)__bfloat16_as_ushort(v[0]) | ((uint32_t)__bfloat16_as_ushort(v[1]) << 16);
    u.y = (uint32_t)__bfloat16_as_ushort(v[2]) | ((uint32_t)__bfloat16_as_ushort(v[3]) << 16);
    *reinterpret_cast<uint2*>(p) = u;
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
  // four consecutive values to a 16-byte aligned address
  __device__ static void store4(T* p, const T (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

struct TcJob {
  int pair0, npairs, out_field, pad;
};

// One GEMM stage of one grid, in device memory (64-byte aligned for the maps).
struct alignas(64) TcGroup {
  CUtensorMap a_hi, a_lo, b_hi, b_lo;  // 3D maps: (K, rows, field | matrix)
  CUtensorMap o_hi, o_lo;              // 4D output maps (inner, outer, a, field) when tma_out
  const TcJob* jobs;
  const short2* pairs;                 // (A field, B matrix)
  void* out_hi;                        // split: hi plane base; f32: float base
  void* out_lo;                        // split: lo plane base
  long long field_elems;               // elements per output field
  long long s_a;                       // output stride of the column index a
  int ldC, n_inner;                    // output row stride and row split (outer, inner)
  int rows, n_a, kblocks, bn, mode, tma_out;
  float alpha;
  int njobs, m_tiles, n_tiles, ntiles;
  int rgroup;                          // row blocks per super-block of the tile order
};

struct TcLaunch {
  const TcGroup* groups;               // device array
  const int* tile0;                    // device prefix sums of group tiles, [ngroups + 1]
  int ngroups, total_tiles;
  int* tile_counter;                   // zeroed before the launch
  int* status;
};

__device__ __forceinline__ void tile_coords(const TcLaunch& L, int tile, int& g, int& j, int& mt, int& nt) {
  int lo = 0, hi = L.ngroups - 1;
  while (lo < hi) {  // last group whose first tile <= tile
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(L.tile0 + mid) <= tile) lo = mid; else hi = mid - 1;
  }
  g = lo;
  const TcGroup& G = L.groups[g];
  int t = tile - __ldg(L.tile0 + g);
  // Tile order: super-blocks of `rgroup` row blocks; inside one, every job
  // in turn over all of its row blocks (column tiles fastest).  rgroup = 1
  // (the default) runs all jobs of one row block back to back, so the A rows
  // they share are read from L2; larger groups make concurrently running
  // tiles write neighbouring rows of one field instead (measured no faster on
  // 160^3-256^3 grids, kept as a compile-time option).
  const int per_sb = G.njobs * G.rgroup * G.n_tiles;
  const int sb = t / per_sb;
  t -= sb * per_sb;
  const int rb0 = sb * G.rgroup;
  const int gsb = min(G.rgroup, G.m_tiles - rb0);  // row blocks in this super-block
  nt = t % G.n_tiles;
  t /= G.n_tiles;
  mt = rb0 + t % gsb;
  j = t / gsb;
}

__device__ __forceinline__ void tc_fail(volatile int* abort, int* status) {
  *abort = 1;
  atomicExch(status, (int)DEMAG_ETIMEOUT);
}

template <class F>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcLaunch L) {
  using T = typename F::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ostage = smem + kStages * kStageBytes;  // epilogue staging (1024-aligned)
  uint64_t* full = reinterpret_cast<uint64_t*>(ostage + kOutStaging);
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
      ptx::mbar_init(&tempty[b], kEpiWarps);
    }
    for (int i = 0; i < kRing; ++i) {
      ptx::mbar_init(&sfull[i], 1);
      ptx::mbar_init(&sempty[i], 1 + kEpiWarps);
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
      int s = 0;
      uint32_t ph = 0;
      int rs = 0;
      uint32_t rph = 0;
      while (!*abort) {
        // take the next tile and hand its id to the MMA and epilogue roles
        if (!ptx::mbar_wait(&sempty[rs], rph ^ 1, abort, kWaitNs)) {
          tc_fail(abort, L.status);
          break;
        }
        const int tile = atomicAdd(L.tile_counter, 1);
        ring[rs] = tile < L.total_tiles ? tile : -1;
        ptx::mbar_arrive(&sfull[rs]);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile >= L.total_tiles) break;
        int g, j, mt, nt;
        tile_coords(L, tile, g, j, mt, nt);
        const TcGroup& G = L.groups[g];
        const TcJob J = G.jobs[j];
        const uint32_t bytes = 2 * kTileA + 2 * (uint32_t)G.bn * kRowBytes;
        for (int pi = 0; pi < J.npairs && !*abort; ++pi) {
          const short2 pr = G.pairs[J.pair0 + pi];
          for (int kb = 0; kb < G.kblocks; ++kb) {
            if (!ptx::mbar_wait(&empty[s], ph ^ 1, abort, kWaitNs)) {
              tc_fail(abort, L.status);
              break;
            }
            uint8_t* st = smem + s * kStageBytes;
            ptx::mbar_arrive_expect_tx(&full[s], bytes);
            ptx::tma_load_3d(st, &G.a_hi, &full[s], kb * F::kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + kTileA, &G.a_lo, &full[s], kb * F::kBK, mt * kBM, pr.x);
            ptx::tma_load_3d(st + 2 * kTileA, &G.b_hi, &full[s], kb * F::kBK, nt * G.bn, pr.y);
            ptx::tma_load_3d(st + 2 * kTileA + kTileB, &G.b_lo, &full[s], kb * F::kBK, nt * G.bn, pr.y);
            if (++s == kStages) { s = 0; ph ^= 1; }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0, tph = 0;
      int buf = 0;
      int rs = 0;
      uint32_t rph = 0;
      while (!*abort) {
        if (!ptx::mbar_wait(&sfull[rs], rph, abort, kWaitNs)) {
          tc_fail(abort, L.status);
          break;
        }
        const int tile = ring[rs];
        ptx::mbar_arrive(&sempty[rs]);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile < 0) break;
        int g, j, mt, nt;
        tile_coords(L, tile, g, j, mt, nt);
        const TcGroup& G = L.groups[g];
        const TcJob J = G.jobs[j];
        const uint32_t idesc = ptx::instr_desc(F::kFormat, kBM, (uint32_t)G.bn);
        const int kblocks = G.kblocks;
        if (!ptx::mbar_wait(&tempty[buf], tph ^ 1, abort, kWaitNs)) {
          tc_fail(abort, L.status);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(buf * kBN);
        uint32_t acc = 0;
        bool ok = true;
        for (int pi = 0; pi < J.npairs && ok; ++pi) {
          for (int kb = 0; kb < kblocks; ++kb) {
            if (!ptx::mbar_wait(&full[s], ph, abort, kWaitNs)) {
              tc_fail(abort, L.status);
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
    const int quad = warp & 3;                // TMEM lane quadrant this warp may access
    const int slice = (warp - 2) / 4;         // which of the quadrant's chunks it takes
    const int rloc = quad * 32 + lane;
    int buf = 0;
    uint32_t tph = 0;
    int rs = 0;
    uint32_t rph = 0;
    uint32_t chunk = 0;  // staged chunks of this warp so far: selects the staging buffer
    while (!*abort) {
      if (!ptx::mbar_wait(&sfull[rs], rph, abort, kWaitNs)) {
        tc_fail(abort, L.status);
        break;
      }
      const int tile = ring[rs];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (tile < 0) break;
      int g, j, mt, nt;
      tile_coords(L, tile, g, j, mt, nt);
      const TcGroup& G = L.groups[g];
      const int out_field = G.jobs[j].out_field;
      if (!ptx::mbar_wait(&tfull[buf], tph, abort, kWaitNs)) {
        tc_fail(abort, L.status);
        break;
      }
      ptx::tc_fence_after();
      const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * kBN);
      const int a0 = nt * G.bn;
      const int bn = G.bn;
      const int n_inner = G.n_inner;
      const int mode = G.mode;
      const float alpha = G.alpha;
      if (G.tma_out) {
        // A warp's 32 rows lie in one `outer` (n_inner % 32 == 0), so each
        // 32-column chunk is one TMA box per plane: stage it in shared memory
        // as [column][row] and store it with the async copy engine.
        const int rw = mt * kBM + quad * 32;
        const int outer_w = rw / n_inner, inner_w = rw - outer_w * n_inner;
        const bool warp_valid = rw < G.rows;
        uint8_t* stg = ostage + (warp - 2) * (kOutBufsPerWarp * kOutBuf);
        for (int c0 = 32 * slice; c0 < bn; c0 += 32 * kEpiSlices) {
          uint32_t r[32];
          ptx::tmem_ld32(taddr + (uint32_t)c0, r);
          ptx::tmem_ld_wait();
          if (!warp_valid) continue;
          // a warp's buffers are used in turn over its whole chunk sequence
          // (across tiles); before reuse, the store that last read a buffer
          // must have finished reading it
          uint8_t* sb = stg + (chunk % kOutBufsPerWarp) * kOutBuf;
          ++chunk;
          if (lane == 0) ptx::bulk_wait_read<kOutBufsPerWarp - 1>();
          __syncwarp();
          if (mode == kOutSplit) {
            T* sh = reinterpret_cast<T*>(sb);
            T* sl = sh + 32 * 32;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              T hi, lo;
              F::split(__uint_as_float(r[jj]), hi, lo);
              sh[jj * 32 + lane] = hi;
              sl[jj * 32 + lane] = lo;
            }
          } else {
            float* sf = reinterpret_cast<float*>(sb);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) sf[jj * 32 + lane] = alpha * __uint_as_float(r[jj]);
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            ptx::tma_store_4d(&G.o_hi, sb, inner_w, outer_w, a0 + c0, out_field);
            if (mode == kOutSplit)
              ptx::tma_store_4d(&G.o_lo, sb + 32 * 32 * sizeof(T), inner_w, outer_w, a0 + c0, out_field);
            ptx::bulk_commit();
          }
        }
      } else {
        const int row = mt * kBM + rloc;
        const bool valid = row < G.rows;
        const int outer = row / n_inner, inner = row - outer * n_inner;
        const long long s_a = G.s_a;
        const long long rbase = (long long)out_field * G.field_elems + (long long)outer * G.ldC + inner;
        const int acount = min(bn, G.n_a - a0);  // columns of this tile that exist
        for (int c0 = 32 * slice; c0 < bn; c0 += 32 * kEpiSlices) {
          uint32_t r[32];
          ptx::tmem_ld32(taddr + (uint32_t)c0, r);
          ptx::tmem_ld_wait();
          if (!valid) continue;
          if (mode == kOutSplit) {
            T* hp = reinterpret_cast<T*>(G.out_hi) + rbase + (long long)(a0 + c0) * s_a;
            T* lp = reinterpret_cast<T*>(G.out_lo) + rbase + (long long)(a0 + c0) * s_a;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              if (c0 + jj < acount) {
                T hi, lo;
                F::split(__uint_as_float(r[jj]), hi, lo);
                *hp = hi;
                *lp = lo;
              }
              hp += s_a;
              lp += s_a;
            }
          } else {
            float* op = reinterpret_cast<float*>(G.out_hi) + rbase + (long long)(a0 + c0) * s_a;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              if (c0 + jj < acount) *op = alpha * __uint_as_float(r[jj]);
              op += s_a;
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
    if (lane == 0) ptx::bulk_wait_all();  // staged stores finished before the block exits
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

// Element-wise kernels over several grids in one launch: item i covers the
// flat range [begin_i, begin_{i+1}) of the launch's index space; a thread's
// indices only grow, so it finds its item by advancing from the last one.
constexpr int kMaxItems = 128;

struct SplitItem {
  const float* x;      // [rows][n] FP32
  void* hi;            // [rows][ld] planes
  void* lo;
  long long begin;     // first flat index of this item
  int n, ld;
  int vec;             // n % 4 == 0 and x 16-byte aligned
};

struct SplitList {
  int count;
  long long total;
  SplitItem it[kMaxItems];
};

// hi/lo split of [rows][n] FP32 tensors into [rows][ld] planes.  The flat
// index space counts groups of four consecutive elements of a row (rows are
// padded to a multiple of four), so a row with n % 4 == 0 moves as 16-byte
// loads and 4-element stores.
template <class F>
__global__ void split_rows_kernel(const __grid_constant__ SplitList L) {
  using T = typename F::T;
  int item = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.total;
       i += (long long)gridDim.x * blockDim.x) {
    while (item + 1 < L.count && i >= L.it[item + 1].begin) ++item;
    const SplitItem& S = L.it[item];
    const int quads = (S.n + 3) >> 2;
    const long long e = i - S.begin;
    const long long r = e / quads;
    const int c = (int)(e - r * quads) * 4;
    const float* src = S.x + r * S.n + c;
    T* hi = reinterpret_cast<T*>(S.hi) + r * S.ld + c;
    T* lo = reinterpret_cast<T*>(S.lo) + r * S.ld + c;
    if (S.vec) {
      const float4 v = *reinterpret_cast<const float4*>(src);
      const float vv[4] = {v.x, v.y, v.z, v.w};
      T h[4], l[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) F::split(vv[j], h[j], l[j]);
      F::store4(hi, h);
      F::store4(lo, l);
    } else {
      for (int j = 0; j < 4 && c + j < S.n; ++j) F::split(src[j], hi[j], lo[j]);
    }
  }
}

// Dense Toeplitz factors of one axis, hi/lo, [M][2][n][ld]; the third axis
// carries the scale c s omega_k.
template <class F>
__global__ void tc_factor_kernel(int M, int glen, int axis, int n, int ld, const double* gen, const double* scale,
                                 typename F::T* hi, typename F::T* lo, const double* fac, size_t tgroup,
                                 size_t toff) {
  const long long total = (long long)M * 2 * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(i % n);
    const long long t = i / n;
    const int ii = (int)(t % n);
    const int kt = (int)(t / n);  // k*2 + type
    // Toeplitz generator (uniform grid) or the full matrix (non-uniform grid)
    double v = fac ? fac[(size_t)kt * tgroup + toff + (size_t)ii * n + jj]
                   : gen[((long long)kt * 3 + axis) * glen + (ii - jj + n - 1)];
    if (axis == 2) v *= scale[kt / 2];
    typename F::T h, l;
    F::split((float)v, h, l);
    const long long o = ((long long)kt * n + ii) * ld + jj;
    hi[o] = h;
    lo[o] = l;
  }
}

// The tensor cores accumulate into TMEM with FP32 additions that do not round
// to nearest, so the error of a long contraction grows with the number of
// MMAs accumulated into one accumulator.  The node-sum stage (2M pairs of
// length n3) is therefore split into groups of at most ~400 accumulations
// (~200 for TF32x3), whose FP32 partial fields are summed on CUDA cores with
// a compensated sum.
static int pairs_per_split(int kblocks, int budget) {
  const int per_pair = kblocks * 6;  // 2 k-steps x 3 products per k-block
  const int pp = budget / (per_pair > 0 ? per_pair : 1);
  return pp < 1 ? 1 : pp;
}

struct ReduceItem {
  const float* part;   // [nout][groups][N] partial fields
  float* out;          // [nout][N]
  long long begin;     // first flat index of this item
  long long N;
  int groups;
  float alpha;
  int vec;             // N % 4 == 0 and out 16-byte aligned: groups of four elements
};

struct ReduceList {
  int count;
  long long total;
  ReduceItem it[kMaxItems];
};

// Neumaier's compensated sum: s + c carries the exact sum of the terms to a
// few ulps for the handful of terms summed here, in round-to-nearest FP32
// arithmetic (the FP64 units of this GPU are too slow to use at memory rate).
struct Csum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float y) {
    const float t = s + y;
    c += fabsf(s) >= fabsf(y) ? (s - t) + y : (y - t) + s;
    s = t;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

// out[q][i] = alpha * sum_g part[q*groups + g][i], compensated; the flat index
// space counts groups of four elements when N % 4 == 0 (16-byte accesses)
__global__ void reduce_parts_kernel(const __grid_constant__ ReduceList L) {
  int item = 0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < L.total;
       idx += (long long)gridDim.x * blockDim.x) {
    while (item + 1 < L.count && idx >= L.it[item + 1].begin) ++item;
    const ReduceItem& R = L.it[item];
    const long long e = idx - R.begin;
    if (R.vec) {
      const long long nq = R.N >> 2;
      const long long q = e / nq, i4 = e - q * nq;
      const float4* src = reinterpret_cast<const float4*>(R.part + q * R.groups * R.N) + i4;
      Csum a[4];
      for (int g = 0; g < R.groups; ++g) {
        const float4 v = src[g * nq];
        a[0].add(v.x);
        a[1].add(v.y);
        a[2].add(v.z);
        a[3].add(v.w);
      }
      reinterpret_cast<float4*>(R.out + q * R.N)[i4] =
          make_float4(R.alpha * a[0].value(), R.alpha * a[1].value(), R.alpha * a[2].value(),
                      R.alpha * a[3].value());
    } else {
      const long long q = e / R.N, i = e - q * R.N;
      const float* src = R.part + q * R.groups * R.N + i;
      Csum a;
      for (int g = 0; g < R.groups; ++g) a.add(src[g * R.N]);
      R.out[e] = R.alpha * a.value();
    }
  }
}

// ---------------------------------------------------------------- short axes on CUDA cores

// A stage whose axis has at most kSmallAxis cells (thin films) would pad both
// the contraction (32-element k-blocks) and the output columns (16-wide tiles)
// on the tensor cores; it runs here instead: one thread per (job, row), the
// job's factor matrices in shared memory (FP32 from the FP64 generators), FP32
// accumulation, the same output layout and hi/lo split as the tensor-core epilogue.
constexpr int kSmallAxis = 16;
constexpr int kSmallChunk = 32;  // factor matrices staged per round (32 x 16 x 16 floats = 32 KB)

struct SmallStage {
  const void* a_hi;
  const void* a_lo;       // input planes: field f, row r at f * a_field + r * a_ld
  long long a_field;
  int a_ld;
  int rows, n, axis;      // rows per field; axis length (contraction and output columns)
  int glen;
  const double* gen;      // [M][2][3][glen]
  const double* fac;      // non-uniform grid: full matrices [M][2][tgroup] (gen unused), else NULL
  long long fac_group, fac_off;  // tgroup and this axis' block offset
  const double* scale;    // [M], applied on the third axis
  const TcJob* jobs;
  const short2* pairs;    // (A field, matrix 2k + type)
  int njobs;
  void* out_hi;
  void* out_lo;
  long long field_elems, s_a;
  int ldC, n_inner, mode;
  float alpha;
};

template <class F>
__global__ void __launch_bounds__(256) small_stage_kernel(const __grid_constant__ SmallStage S) {
  using T = typename F::T;
  __shared__ float sB[kSmallChunk * kSmallAxis * kSmallAxis];
  const TcJob J = S.jobs[blockIdx.y];
  const int n = S.n;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = row < S.rows;
  float acc[kSmallAxis];
#pragma unroll
  for (int a = 0; a < kSmallAxis; ++a) acc[a] = 0.f;
  for (int p0 = 0; p0 < J.npairs; p0 += kSmallChunk) {
    const int np = min(kSmallChunk, J.npairs - p0);
    __syncthreads();  // the previous round's matrices are consumed
    for (int i = threadIdx.x; i < np * n * n; i += blockDim.x) {
      const int p = i / (n * n), rem = i - p * n * n;
      const int a = rem / n, kk = rem - a * n;
      const short2 pr = S.pairs[J.pair0 + p0 + p];
      const int k = pr.y >> 1;
      double v = S.fac ? S.fac[(long long)pr.y * S.fac_group + S.fac_off + (long long)a * n + kk]
                       : S.gen[((long long)pr.y * 3 + S.axis) * S.glen + (a - kk + n - 1)];
      if (S.axis == 2) v *= S.scale[k];
      sB[i] = (float)v;
    }
    __syncthreads();
    if (!valid) continue;
    for (int p = 0; p < np; ++p) {
      const short2 pr = S.pairs[J.pair0 + p0 + p];
      const long long off = (long long)pr.x * S.a_field + (long long)row * S.a_ld;
      const T* hi = reinterpret_cast<const T*>(S.a_hi) + off;
      const T* lo = reinterpret_cast<const T*>(S.a_lo) + off;
      float x[kSmallAxis];
#pragma unroll
      for (int kk = 0; kk < kSmallAxis; ++kk) x[kk] = kk < n ? (float)hi[kk] + (float)lo[kk] : 0.f;
      const float* b = sB + p * n * n;
#pragma unroll
      for (int a = 0; a < kSmallAxis; ++a) {
        if (a >= n) break;
        float t = acc[a];
#pragma unroll
        for (int kk = 0; kk < kSmallAxis; ++kk)
          if (kk < n) t = fmaf(b[a * n + kk], x[kk], t);
        acc[a] = t;
      }
    }
  }
  if (!valid) return;
  const int outer = row / S.n_inner, inner = row - outer * S.n_inner;
  const long long rbase = (long long)J.out_field * S.field_elems + (long long)outer * S.ldC + inner;
#pragma unroll
  for (int a = 0; a < kSmallAxis; ++a) {
    if (a >= n) break;
    if (S.mode == kOutSplit) {
      T h, l;
      F::split(acc[a], h, l);
      reinterpret_cast<T*>(S.out_hi)[rbase + a * S.s_a] = h;
      reinterpret_cast<T*>(S.out_lo)[rbase + a * S.s_a] = l;
    } else {
      reinterpret_cast<float*>(S.out_hi)[rbase + a * S.s_a] = S.alpha * acc[a];
    }
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

// 4D map over an output field set: (inner, outer, a, field) with the given
// strides in elements; box (32, 1, 32, 1) = one epilogue warp's 32 rows x 32
// output columns, no swizzle.
static bool make_out_map(CUtensorMap* m, void* base, int elem_bytes, uint64_t inner, uint64_t outer, uint64_t na,
                         uint64_t fields, uint64_t ld, uint64_t s_a, uint64_t field_elems) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[4] = {inner, outer, na, fields};
  cuuint64_t strides[3] = {ld * elem_bytes, s_a * elem_bytes, field_elems * elem_bytes};
  cuuint32_t box[4] = {32, 1, 32, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Stage programs of a plan: forward stages 0-2, adjoint stages 3-5.
enum { kFwd1 = 0, kFwd2, kFwd3, kAdj1, kAdj2, kAdj3, kPrograms };

// Per-plan, per-form tensor-core state.
struct TcState {
  int elem;               // bytes per element (2 BF16, 4 TF32)
  int ld[3];              // padded row lengths (16-byte multiples)
  int bn[3];              // N tile width per axis
  void* B[3][2];          // per axis: hi / lo factors [M][2][n][ld]
  void* X[2];             // split input: [3][n3 n2][ld1]
  void* buf1[2];          // [3M][n1 n3][ld2]
  void* buf2[2];          // [3M][n2 n1][ld3]
  int* status;
  int* counter;           // dynamic tile counter of the running launch
  float* part;            // split node-sum partial fields
  int pp3;                // (A, B) pairs per accumulator in the node-sum stage
  int part_fields;        // partial fields allocated
  int groups_fwd, groups_adj;  // partial fields used by the forward / adjoint node sum
  int tma[3];             // stage epilogue stores through TMA
  // stage programs: the group descriptors (device) and their job / pair tables
  TcGroup* prog;          // device [kPrograms]
  TcJob* jobs;            // device, all programs
  short2* pairs;          // device, all programs
  int* tile0;             // device [kPrograms][2]: {0, ntiles} for single-group launches
  TcGroup host_prog[kPrograms];
  bool small[kPrograms];          // program runs on CUDA cores (axis of at most kSmallAxis cells)
  SmallStage small_prog[kPrograms];
  // analytic stray field: the forward stage programs with the derivative
  // factors of their axis (built on first use)
  bool field_ready;
  void* Bd[3][2];                 // per axis: hi / lo derivative factors [M][2][n][ld]
  TcGroup dprog_host[3];
  TcGroup* dprog;                 // device [3]
  int* dtile0;                    // device [3][2]
  SmallStage small_dprog[3];
  size_t bytes;
};

// Grouped descriptors of the forward stages of several plans (one launch per
// stage over all of them); owned by a plan's cache or by a captured graph.
struct TcBatch {
  std::vector<demag_plan*> plans;
  std::vector<unsigned long long> serials;  // with the pointers, the cache key
  int prec = -1;
  TcGroup* groups = nullptr;           // device [3][count]
  int* tile0 = nullptr;                // device [3][count + 1]
  int total[3] = {0, 0, 0};
};

struct TcHolder {
  TcState* s[2] = {nullptr, nullptr};  // [0] BF16x3, [1] TF32x3
  TcBatch* cache = nullptr;            // last plan list given to demag_apply_full_batched
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
  cudaFree(S->prog);
  cudaFree(S->jobs);
  cudaFree(S->pairs);
  cudaFree(S->tile0);
  for (int p = 0; p < 3; ++p)
    for (int h = 0; h < 2; ++h) cudaFree(S->Bd[p][h]);
  cudaFree(S->dprog);
  cudaFree(S->dtile0);
  delete S;
}

void tc_destroy(demag_plan* P) {
  TcHolder* H = reinterpret_cast<TcHolder*>(P->tc);
  if (!H) return;
  for (auto*& s : H->s) {
    free_state(s);
    s = nullptr;
  }
  tc_batch_destroy(H->cache);
  delete H;
  P->tc = nullptr;
}

static int grid_blocks(long long count) {
  long long b = (count + 255) / 256;
  return (int)(b > 152 * 16 ? 152 * 16 : (b < 1 ? 1 : b));
}

static TcJob job(int pair0, int npairs, int out_field) {
  TcJob j;
  j.pair0 = pair0;
  j.npairs = npairs;
  j.out_field = out_field;
  j.pad = 0;
  return j;
}

// matrix index of (node k, type) in the per-axis factor maps
static short mat(int k, int type) { return (short)(2 * k + type); }

// Build the six stage programs of a plan (host descriptors, job and pair tables).
struct ProgramBuild {
  std::vector<TcJob> jobs;
  std::vector<short2> pairs;
  int job0[kPrograms], pair0[kPrograms];
};

static void set_stage(TcGroup& G, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
                      const CUtensorMap& blo, int rows, int n_a, int K, int bk, int bn, void* out_hi, void* out_lo,
                      long long field_elems, long long s_a, int ldC, int n_inner, int mode, float alpha) {
  G.a_hi = ahi;
  G.a_lo = alo;
  G.b_hi = bhi;
  G.b_lo = blo;
  G.rows = rows;
  G.n_a = n_a;
  G.kblocks = (K + bk - 1) / bk;
  G.bn = bn;
  G.out_hi = out_hi;
  G.out_lo = out_lo;
  G.field_elems = field_elems;
  G.s_a = s_a;
  G.ldC = ldC;
  G.n_inner = n_inner;
  G.mode = mode;
  G.alpha = alpha;
  G.m_tiles = (rows + kBM - 1) / kBM;
  G.rgroup = kRowGroup < G.m_tiles ? kRowGroup : G.m_tiles;
  G.n_tiles = (n_a + bn - 1) / bn;
}

static demag_status build_programs(demag_plan* P, TcState* S, const CUtensorMap (&mapX)[2],
                                   const CUtensorMap (&map1)[2], const CUtensorMap (&map2)[2],
                                   const CUtensorMap (&mapB)[3][2], const CUtensorMap (&out1)[2],
                                   const CUtensorMap (&out2)[2], const CUtensorMap& out3, int bk,
                                   cudaStream_t st) {
  const int n1 = P->n[0], n2 = P->n[1], n3 = P->n[2], M = P->M;
  const long long N = (long long)n1 * n2 * n3;
  ProgramBuild b;
  auto begin = [&](int prog) {
    b.job0[prog] = (int)b.jobs.size();
    b.pair0[prog] = (int)b.pairs.size();
  };
  auto add_job = [&](int prog, int npairs, int out_field) {
    b.jobs.push_back(job((int)b.pairs.size() - b.pair0[prog] - npairs, npairs, out_field));
  };
  // forward mode 1: Y[k][q] = m_q x_1 T_{k,q,1}; rows (i3, i2), contraction i1 -> Y [i1'][i3][i2]
  begin(kFwd1);
  for (int q = 0; q < 3; ++q)
    for (int k = 0; k < M; ++k) {
      b.pairs.push_back(make_short2((short)q, mat(k, q == 0 ? 1 : 0)));
      add_job(kFwd1, 1, 3 * k + q);
    }
  // forward mode 2: U_k = Y_k1 x_2 E + Y_k2 x_2 F, V_k = Y_k3 x_2 E; rows (i1', i3) -> [i2'][i1'][i3]
  begin(kFwd2);
  for (int k = 0; k < M; ++k) {
    b.pairs.push_back(make_short2((short)(3 * k + 0), mat(k, 0)));
    b.pairs.push_back(make_short2((short)(3 * k + 1), mat(k, 1)));
    add_job(kFwd2, 2, 2 * k);
    b.pairs.push_back(make_short2((short)(3 * k + 2), mat(k, 0)));
    add_job(kFwd2, 1, 2 * k + 1);
  }
  // forward mode 3, node sum split in groups of pp3 pairs: part_g = sum U_k x_3 S E + V_k x_3 S F
  begin(kFwd3);
  for (int k = 0; k < M; ++k) {
    b.pairs.push_back(make_short2((short)(2 * k), mat(k, 0)));
    b.pairs.push_back(make_short2((short)(2 * k + 1), mat(k, 1)));
  }
  S->groups_fwd = (2 * M + S->pp3 - 1) / S->pp3;
  for (int g = 0; g < S->groups_fwd; ++g) {
    const int p0 = g * S->pp3;
    const int np = (2 * M - p0) < S->pp3 ? (2 * M - p0) : S->pp3;
    b.jobs.push_back(job(p0, np, g));
  }
  // adjoint mode 1: Ya_k = y x_1 F, Yb_k = y x_1 E  (fields 2k, 2k+1 of buf1)
  begin(kAdj1);
  for (int k = 0; k < M; ++k)
    for (int t = 0; t < 2; ++t) {
      b.pairs.push_back(make_short2((short)0, mat(k, t == 0 ? 1 : 0)));
      add_job(kAdj1, 1, 2 * k + t);
    }
  // adjoint mode 2: Za = Ya x_2 E (g1), Zb = Yb x_2 F (g2), Zc = Yb x_2 E (g3)  (fields 3k+q of buf2)
  begin(kAdj2);
  for (int k = 0; k < M; ++k) {
    const short src[3] = {(short)(2 * k), (short)(2 * k + 1), (short)(2 * k + 1)};
    const int typ[3] = {0, 1, 0};
    for (int q = 0; q < 3; ++q) {
      b.pairs.push_back(make_short2(src[q], mat(k, typ[q])));
      add_job(kAdj2, 1, 3 * k + q);
    }
  }
  // adjoint mode 3 with the node sum split: part_{q,g} = sum_k Z_kq x_3 S T_{k,q,3}
  begin(kAdj3);
  S->groups_adj = (M + S->pp3 - 1) / S->pp3;
  for (int q = 0; q < 3; ++q) {
    const int base = (int)b.pairs.size() - b.pair0[kAdj3];
    for (int k = 0; k < M; ++k) b.pairs.push_back(make_short2((short)(3 * k + q), mat(k, q == 2 ? 1 : 0)));
    for (int gi = 0; gi < S->groups_adj; ++gi) {
      const int p0 = gi * S->pp3;
      const int np = (M - p0) < S->pp3 ? (M - p0) : S->pp3;
      b.jobs.push_back(job(base + p0, np, q * S->groups_adj + gi));
    }
  }
  const int job_end = (int)b.jobs.size();

  const long long f1 = (long long)n1 * n3 * S->ld[1], f2 = (long long)n2 * n1 * S->ld[2];
  TcGroup* H = S->host_prog;
  memset(H, 0, sizeof(S->host_prog));
  set_stage(H[kFwd1], mapX[0], mapX[1], mapB[0][0], mapB[0][1], n3 * n2, n1, n1, bk, S->bn[0], S->buf1[0],
            S->buf1[1], f1, (long long)n3 * S->ld[1], S->ld[1], n2, kOutSplit, 1.f);
  set_stage(H[kFwd2], map1[0], map1[1], mapB[1][0], mapB[1][1], n1 * n3, n2, n2, bk, S->bn[1], S->buf2[0],
            S->buf2[1], f2, (long long)n1 * S->ld[2], S->ld[2], n3, kOutSplit, 1.f);
  set_stage(H[kFwd3], map2[0], map2[1], mapB[2][0], mapB[2][1], n2 * n1, n3, n3, bk, S->bn[2], S->part, nullptr, N,
            (long long)n2 * n1, n1, n1, kOutF32, 1.f);
  H[kAdj1] = H[kFwd1];
  H[kAdj2] = H[kFwd2];
  H[kAdj3] = H[kFwd3];
  for (int p = 0; p < kPrograms; ++p) {
    const int stage = p % 3;
    if (S->tma[stage]) {
      H[p].tma_out = 1;
      if (stage == 0) { H[p].o_hi = out1[0]; H[p].o_lo = out1[1]; }
      if (stage == 1) { H[p].o_hi = out2[0]; H[p].o_lo = out2[1]; }
      if (stage == 2) H[p].o_hi = out3;
    }
  }
  // job and pair tables
  DEMAG_CUDA(P, cudaMalloc(&S->jobs, sizeof(TcJob) * b.jobs.size()));
  DEMAG_CUDA(P, cudaMalloc(&S->pairs, sizeof(short2) * b.pairs.size()));
  DEMAG_CUDA(P, cudaMemcpy(S->jobs, b.jobs.data(), sizeof(TcJob) * b.jobs.size(), cudaMemcpyHostToDevice));
  DEMAG_CUDA(P, cudaMemcpy(S->pairs, b.pairs.data(), sizeof(short2) * b.pairs.size(), cudaMemcpyHostToDevice));
  for (int p = 0; p < kPrograms; ++p) {
    const int jend = p + 1 < kPrograms ? b.job0[p + 1] : job_end;
    H[p].jobs = S->jobs + b.job0[p];
    H[p].pairs = S->pairs + b.pair0[p];
    H[p].njobs = jend - b.job0[p];
    H[p].ntiles = H[p].njobs * H[p].m_tiles * H[p].n_tiles;
  }
  // stages along an axis of at most kSmallAxis cells run on CUDA cores
  {
    const void* in_hi[3] = {S->X[0], S->buf1[0], S->buf2[0]};
    const void* in_lo[3] = {S->X[1], S->buf1[1], S->buf2[1]};
    const long long rows_of[3] = {(long long)n3 * n2, (long long)n1 * n3, (long long)n2 * n1};
    for (int p = 0; p < kPrograms; ++p) {
      const int stage = p % 3;
      S->small[p] = P->n[stage] <= kSmallAxis;
      if (!S->small[p]) continue;
      SmallStage& Q = S->small_prog[p];
      const TcGroup& G = H[p];
      Q.a_hi = in_hi[stage];
      Q.a_lo = in_lo[stage];
      Q.a_ld = S->ld[stage];
      Q.a_field = rows_of[stage] * S->ld[stage];
      Q.rows = G.rows;
      Q.n = P->n[stage];
      Q.axis = stage;
      Q.glen = P->glen;
      Q.gen = P->gen64;
      Q.fac = P->fac64;
      Q.fac_group = (long long)P->tgroup;
      Q.fac_off = (long long)P->toff[stage];
      Q.scale = P->scale;
      Q.jobs = G.jobs;
      Q.pairs = G.pairs;
      Q.njobs = G.njobs;
      Q.out_hi = G.out_hi;
      Q.out_lo = G.out_lo;
      Q.field_elems = G.field_elems;
      Q.s_a = G.s_a;
      Q.ldC = G.ldC;
      Q.n_inner = G.n_inner;
      Q.mode = G.mode;
      Q.alpha = G.alpha;
    }
  }
  DEMAG_CUDA(P, cudaMalloc(&S->prog, sizeof(TcGroup) * kPrograms));
  DEMAG_CUDA(P, cudaMemcpy(S->prog, H, sizeof(TcGroup) * kPrograms, cudaMemcpyHostToDevice));
  int t0[2 * kPrograms];
  for (int p = 0; p < kPrograms; ++p) {
    t0[2 * p] = 0;
    t0[2 * p + 1] = H[p].ntiles;
  }
  DEMAG_CUDA(P, cudaMalloc(&S->tile0, sizeof(t0)));
  DEMAG_CUDA(P, cudaMemcpy(S->tile0, t0, sizeof(t0), cudaMemcpyHostToDevice));
  (void)st;
  return DEMAG_OK;
}

template <class F>
static demag_status prepare_form(demag_plan* P, TcState* S, cudaStream_t st) {
  const int M = P->M;
  for (int p = 0; p < 3; ++p) {
    long long total = (long long)M * 2 * P->n[p] * P->n[p];
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<F><<<grid_blocks(total), 256, 0, st>>>(
                     M, P->glen, p, P->n[p], S->ld[p], P->gen64, P->scale, (typename F::T*)S->B[p][0],
                     (typename F::T*)S->B[p][1], P->fac64, P->tgroup, P->toff[p]));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  static unsigned long long attr = 0;  // devices whose kernel attribute is set
  int dev = 0;
  DEMAG_CUDA(P, cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr & bit)) {
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_gemm_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
    attr |= bit;
  }
  return DEMAG_OK;
}

template <class F>
static demag_status run_program(demag_plan* P, TcState* S, int prog, cudaStream_t st);

// Point stage program `prog` at output-column tile width bn (device copy included).
static demag_status set_tile_width(demag_plan* P, TcState* S, int prog, int bn) {
  TcGroup& G = S->host_prog[prog];
  const int axis = prog % 3;
  const int M = P->M;
  for (int h = 0; h < 2; ++h)
    if (!make_map(h ? &G.b_lo : &G.b_hi, S->B[axis][h], S->elem, P->n[axis], P->n[axis], 2 * M, S->ld[axis], bn))
      return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  G.bn = bn;
  G.n_tiles = (G.n_a + bn - 1) / bn;
  G.ntiles = G.njobs * G.m_tiles * G.n_tiles;
  const int t0[2] = {0, G.ntiles};
  DEMAG_CUDA(P, cudaMemcpy(S->prog + prog, &G, sizeof(TcGroup), cudaMemcpyHostToDevice));
  DEMAG_CUDA(P, cudaMemcpy(S->tile0 + 2 * prog, t0, sizeof(t0), cudaMemcpyHostToDevice));
  return DEMAG_OK;
}

// Autotuning of the output-column tile width of every stage program: the
// default (256, or the column count rounded up to 16) and 128 and 64 below it
// are timed (one warm-up, three timed launches, operands as they are in the
// workspace), and the fastest is kept.
template <class F>
static demag_status tune_tile_widths(demag_plan* P, TcState* S, cudaStream_t st) {
  cudaEvent_t e0, e1;
  DEMAG_CUDA(P, cudaEventCreate(&e0));
  DEMAG_CUDA(P, cudaEventCreate(&e1));
  demag_status s = DEMAG_OK;
  for (int prog = 0; prog < kPrograms && s == DEMAG_OK; ++prog) {
    if (S->small[prog]) continue;  // runs on CUDA cores
    const int def = S->host_prog[prog].bn;
    std::vector<int> cands{def};
    for (int c = 128; c >= 64; c /= 2)
      if (c < def) cands.push_back(c);
    if (cands.size() == 1) continue;
    float best = 1e30f;
    int best_bn = def;
    for (int c : cands) {
      s = set_tile_width(P, S, prog, c);
      if (s == DEMAG_OK) s = run_program<F>(P, S, prog, st);
      if (s != DEMAG_OK) break;
      DEMAG_CUDA(P, cudaEventRecord(e0, st));
      for (int r = 0; r < 3 && s == DEMAG_OK; ++r) s = run_program<F>(P, S, prog, st);
      DEMAG_CUDA(P, cudaEventRecord(e1, st));
      DEMAG_CUDA(P, cudaEventSynchronize(e1));
      if (s != DEMAG_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_bn = c;
      }
    }
    if (s == DEMAG_OK) s = set_tile_width(P, S, prog, best_bn);
    if (s == DEMAG_OK) {
      demag_plan::Tuned t;
      t.kind = S->elem == 2 ? 1 : 2;
      t.key[0] = prog;
      t.key[1] = def;
      t.key[2] = 0;
      t.value = best_bn;
      t.ms = best / 3.f;
      P->tuned.push_back(t);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == DEMAG_OK) s = tc_sync_status(P, st);
  return s;
}

demag_status tc_prepare(demag_plan* P, demag_precision prec, cudaStream_t st) {
  if (prec != DEMAG_BF16X3 && prec != DEMAG_TF32X3)
    return set_error(P, DEMAG_EUNSUPPORTED, "tensor-core form %d is not built", (int)prec);
  if (state(P, prec)) return DEMAG_OK;
  if (!encode_fn()) return set_error(P, DEMAG_ECUDA, "cuTensorMapEncodeTiled is unavailable");
  if (!P->tc) P->tc = new TcHolder();
  TcHolder* Hd = reinterpret_cast<TcHolder*>(P->tc);
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
    // TF32x3 issues twice the MMAs per K of BF16x3 in stages 1-2 as well, so its
    // node sum gets half the accumulation budget
    S->pp3 = pairs_per_split(kb3, S->elem == 4 ? 200 : 400);
    // a node-sum stage on CUDA cores accumulates in round-to-nearest FP32; its
    // groups only split the work (one job per group) over more blocks
    if (n3 <= kSmallAxis) S->pp3 = std::min(S->pp3, 4);
    const int gf = (2 * M + S->pp3 - 1) / S->pp3;   // forward: 2M pairs in one sum
    const int ga = (M + S->pp3 - 1) / S->pp3;       // adjoint: M pairs per component
    const int fields = gf > 3 * ga ? gf : 3 * ga;
    S->part_fields = fields;
    ok = ok && alloc((void**)&S->part, sizeof(float) * (size_t)fields * n1 * n2 * n3);
  }
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ENOMEM, "tensor-core workspace allocation failed");
  }
  CUtensorMap mapB[3][2], mapX[2], map1[2], map2[2], out1[2], out2[2], out3;
  memset(mapB, 0, sizeof(mapB));  // maps of CUDA-core stages stay unset
  memset(mapX, 0, sizeof(mapX));
  memset(map1, 0, sizeof(map1));
  memset(map2, 0, sizeof(map2));
  memset(out1, 0, sizeof(out1));
  memset(out2, 0, sizeof(out2));
  memset(&out3, 0, sizeof(out3));
  for (int h = 0; h < 2; ++h) {
    for (int p = 0; p < 3; ++p)
      if (P->n[p] > kSmallAxis)
        ok = ok && make_map(&mapB[p][h], S->B[p][h], S->elem, P->n[p], P->n[p], 2 * M, S->ld[p], S->bn[p]);
    if (n1 > kSmallAxis) ok = ok && make_map(&mapX[h], S->X[h], S->elem, n1, (uint64_t)n3 * n2, 3, S->ld[0], kBM);
    if (n2 > kSmallAxis)
      ok = ok && make_map(&map1[h], S->buf1[h], S->elem, n2, (uint64_t)n1 * n3, 3 * M, S->ld[1], kBM);
    if (n3 > kSmallAxis)
      ok = ok && make_map(&map2[h], S->buf2[h], S->elem, n3, (uint64_t)n2 * n1, 3 * M, S->ld[2], kBM);
  }
  // epilogue stores through TMA where a warp's 32 output rows share one outer
  // index (n_inner % 32 == 0) and a 32 x 32 chunk fits the staging buffer
  // (BF16 planes, FP32 partials)
  S->tma[0] = (n2 % 32 == 0) && S->elem == 2;
  S->tma[1] = (n3 % 32 == 0) && S->elem == 2;
  S->tma[2] = (n1 % 32 == 0);
  for (int h = 0; h < 2; ++h) {
    if (S->tma[0])
      ok = ok && make_out_map(&out1[h], S->buf1[h], S->elem, n2, n3, n1, 3 * M, S->ld[1], (uint64_t)n3 * S->ld[1],
                              (uint64_t)n1 * n3 * S->ld[1]);
    if (S->tma[1])
      ok = ok && make_out_map(&out2[h], S->buf2[h], S->elem, n3, n1, n2, 3 * M, S->ld[2], (uint64_t)n1 * S->ld[2],
                              (uint64_t)n2 * n1 * S->ld[2]);
  }
  if (S->tma[2])
    ok = ok && make_out_map(&out3, S->part, 4, n1, n2, n3, S->part_fields, n1, (uint64_t)n2 * n1,
                            (uint64_t)n1 * n2 * n3);
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  }
  const int bk = kRowBytes / S->elem;
  demag_status s = build_programs(P, S, mapX, map1, map2, mapB, out1, out2, out3, bk, st);
  if (s == DEMAG_OK)
    s = prec == DEMAG_TF32X3 ? prepare_form<Tf32Form>(P, S, st) : prepare_form<Bf16Form>(P, S, st);
  if (s == DEMAG_OK && P->autotune) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (cap == cudaStreamCaptureStatusNone) {
      Hd->s[form_index(prec)] = S;  // tc_sync_status reads the state through the holder
      s = prec == DEMAG_TF32X3 ? tune_tile_widths<Tf32Form>(P, S, st) : tune_tile_widths<Bf16Form>(P, S, st);
      Hd->s[form_index(prec)] = nullptr;
    }
  }
  if (s != DEMAG_OK) {
    free_state(S);
    return s;
  }
  Hd->s[form_index(prec)] = S;
  return DEMAG_OK;
}

template <class F>
static demag_status launch_groups(demag_plan* P, const TcGroup* groups, const int* tile0, int ngroups,
                                  int total_tiles, int* counter, int* status, cudaStream_t st) {
  if (total_tiles <= 0) return DEMAG_OK;
  TcLaunch L;
  L.groups = groups;
  L.tile0 = tile0;
  L.ngroups = ngroups;
  L.total_tiles = total_tiles;
  L.tile_counter = counter;
  L.status = status;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = total_tiles < sms ? total_tiles : sms;
  DEMAG_CUDA(P, cudaMemsetAsync(counter, 0, sizeof(int), st));
  DEMAG_LAUNCH(P, kFamGemmTc, st, tc_gemm_kernel<F><<<grid, kTcThreads, kSmemBytes, st>>>(L));
  DEMAG_LAUNCHED(P, "tc_gemm_kernel");
  return DEMAG_OK;
}

template <class F>
static demag_status launch_small(demag_plan* P, const SmallStage& Q, cudaStream_t st) {
  const dim3 grid((unsigned)((Q.rows + 255) / 256), (unsigned)Q.njobs);
  DEMAG_LAUNCH(P, kFamGemmSimt, st, small_stage_kernel<F><<<grid, 256, 0, st>>>(Q));
  DEMAG_LAUNCHED(P, "small_stage_kernel");
  return DEMAG_OK;
}

template <class F>
static demag_status run_program(demag_plan* P, TcState* S, int prog, cudaStream_t st) {
  if (S->small[prog]) return launch_small<F>(P, S->small_prog[prog], st);
  return launch_groups<F>(P, S->prog + prog, S->tile0 + 2 * prog, 1, S->host_prog[prog].ntiles, S->counter,
                          S->status, st);
}

template <class F>
static demag_status launch_split(demag_plan* P, const SplitList& L, cudaStream_t st) {
  DEMAG_LAUNCH(P, kFamSplit, st, split_rows_kernel<F><<<grid_blocks(L.total), 256, 0, st>>>(L));
  DEMAG_LAUNCHED(P, "split_rows_kernel");
  return DEMAG_OK;
}

static void add_split(SplitList& L, demag_plan* P, TcState* S, const float* x, int fields) {
  SplitItem& it = L.it[L.count++];
  it.x = x;
  it.hi = S->X[0];
  it.lo = S->X[1];
  it.begin = L.total;
  it.n = P->n[0];
  it.ld = S->ld[0];
  it.vec = (P->n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0);
  L.total += (long long)fields * P->n[2] * P->n[1] * ((P->n[0] + 3) / 4);
}

template <class F>
static demag_status split_input(demag_plan* P, TcState* S, const float* x, int fields, cudaStream_t st) {
  SplitList L;
  L.count = 0;
  L.total = 0;
  add_split(L, P, S, x, fields);
  return launch_split<F>(P, L, st);
}

static demag_status launch_reduce(demag_plan* P, const ReduceList& L, cudaStream_t st) {
  DEMAG_LAUNCH(P, kFamMisc, st, reduce_parts_kernel<<<grid_blocks(L.total), 256, 0, st>>>(L));
  DEMAG_LAUNCHED(P, "reduce_parts_kernel");
  return DEMAG_OK;
}

static void add_reduce(ReduceList& L, demag_plan* P, TcState* S, int groups, int nout, float alpha, float* out) {
  const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
  ReduceItem& it = L.it[L.count++];
  it.part = S->part;
  it.out = out;
  it.begin = L.total;
  it.N = N;
  it.groups = groups;
  it.alpha = alpha;
  it.vec = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
  L.total += it.vec ? nout * (N >> 2) : nout * N;
}

static demag_status reduce_parts(demag_plan* P, TcState* S, int groups, int nout, float alpha, float* out,
                                 cudaStream_t st) {
  ReduceList L;
  L.count = 0;
  L.total = 0;
  add_reduce(L, P, S, groups, nout, alpha, out);
  return launch_reduce(P, L, st);
}

template <class F>
static demag_status forward_chain(demag_plan* P, TcState* S, const float* m, float* phi, cudaStream_t st) {
  demag_status s = split_input<F>(P, S, m, 3, st);
  for (int prog = kFwd1; prog <= kFwd3 && s == DEMAG_OK; ++prog) s = run_program<F>(P, S, prog, st);
  if (s != DEMAG_OK) return s;
  return reduce_parts(P, S, S->groups_fwd, 1, 1.f, phi, st);
}

template <class F>
static demag_status adjoint_chain(demag_plan* P, TcState* S, const float* y, float* g, cudaStream_t st) {
  demag_status s = split_input<F>(P, S, y, 1, st);
  for (int prog = kAdj1; prog <= kAdj3 && s == DEMAG_OK; ++prog) s = run_program<F>(P, S, prog, st);
  if (s != DEMAG_OK) return s;
  return reduce_parts(P, S, S->groups_adj, 3, -1.f, g, st);
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

void tc_batch_destroy(TcBatch* B) {
  if (!B) return;
  cudaFree(B->groups);
  cudaFree(B->tile0);
  delete B;
}

// Concatenate the forward stage programs of `plans` (which must be distinct and
// have their tensor-core state for `prec`) into per-stage group arrays.
demag_status tc_batch_create(demag_plan* const* plans, int count, demag_precision prec, TcBatch** out) {
  *out = nullptr;
  demag_plan* P0 = plans[0];
  TcBatch* B = new TcBatch();
  B->plans.assign(plans, plans + count);
  for (int i = 0; i < count; ++i) B->serials.push_back(plans[i]->serial);
  B->prec = (int)prec;
  // largest grids first: the dynamic tile counter then hands out their long
  // tile streams early and the small grids' tiles fill the tail of the launch
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto cells = [&](int i) { return (long long)plans[i]->n[0] * plans[i]->n[1] * plans[i]->n[2]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cells(a) > cells(b); });
  std::vector<TcGroup> g(3 * (size_t)count);
  std::vector<int> t0(3 * (size_t)(count + 1));
  for (int st3 = 0; st3 < 3; ++st3) {
    int acc = 0;
    for (int i = 0; i < count; ++i) {
      const TcState* S = state(plans[order[i]], prec);
      g[st3 * count + i] = S->host_prog[kFwd1 + st3];
      t0[st3 * (count + 1) + i] = acc;
      // a stage that runs on CUDA cores keeps its slot with no tiles
      if (!S->small[kFwd1 + st3]) acc += S->host_prog[kFwd1 + st3].ntiles;
    }
    t0[st3 * (count + 1) + count] = acc;
    B->total[st3] = acc;
  }
  if (cudaMalloc(&B->groups, sizeof(TcGroup) * g.size()) != cudaSuccess ||
      cudaMalloc(&B->tile0, sizeof(int) * t0.size()) != cudaSuccess) {
    tc_batch_destroy(B);
    return set_error(P0, DEMAG_ENOMEM, "grouped launch descriptors: allocation failed");
  }
  cudaError_t e = cudaMemcpy(B->groups, g.data(), sizeof(TcGroup) * g.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B->tile0, t0.data(), sizeof(int) * t0.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tc_batch_destroy(B);
    return cuda_error(P0, e, "grouped launch descriptors");
  }
  *out = B;
  return DEMAG_OK;
}

// Several grids in one call: each plan's input is split, then every forward
// stage of all grids runs as ONE persistent launch over the concatenated group
// descriptors (tiles of all grids share the dynamic tile counter of the first
// plan), then each plan's node-sum partials are reduced into its phi.
template <class F>
static demag_status batched_chain(const TcBatch* B, const float* const* m, float* const* phi, cudaStream_t st) {
  const demag_precision prec = (demag_precision)B->prec;
  const int count = (int)B->plans.size();
  demag_plan* P0 = B->plans[0];
  TcState* S0 = state(P0, prec);
  // one split launch per kMaxItems grids
  for (int i0 = 0; i0 < count; i0 += kMaxItems) {
    SplitList L;
    L.count = 0;
    L.total = 0;
    for (int i = i0; i < count && i < i0 + kMaxItems; ++i) add_split(L, B->plans[i], state(B->plans[i], prec), m[i], 3);
    demag_status s = launch_split<F>(P0, L, st);
    if (s != DEMAG_OK) return s;
  }
  for (int st3 = 0; st3 < 3; ++st3) {
    demag_status s = launch_groups<F>(P0, B->groups + (size_t)st3 * count, B->tile0 + (size_t)st3 * (count + 1),
                                      count, B->total[st3], S0->counter, S0->status, st);
    for (int i = 0; i < count && s == DEMAG_OK; ++i) {
      TcState* S = state(B->plans[i], prec);
      if (S->small[kFwd1 + st3]) s = launch_small<F>(B->plans[i], S->small_prog[kFwd1 + st3], st);
    }
    if (s != DEMAG_OK) return s;
  }
  for (int i0 = 0; i0 < count; i0 += kMaxItems) {
    ReduceList L;
    L.count = 0;
    L.total = 0;
    for (int i = i0; i < count && i < i0 + kMaxItems; ++i) {
      TcState* S = state(B->plans[i], prec);
      add_reduce(L, B->plans[i], S, S->groups_fwd, 1, 1.f, phi[i]);
    }
    demag_status s = launch_reduce(P0, L, st);
    if (s != DEMAG_OK) return s;
  }
  return DEMAG_OK;
}

demag_status tc_batch_run(const TcBatch* B, const float* const* m, float* const* phi, cudaStream_t st) {
  return B->prec == DEMAG_TF32X3 ? batched_chain<Tf32Form>(B, m, phi, st) : batched_chain<Bf16Form>(B, m, phi, st);
}

demag_status tc_forward_batched(demag_plan* const* plans, const float* const* m, float* const* phi, int count,
                                demag_precision prec, cudaStream_t st) {
  if (count <= 0) return DEMAG_OK;
  TcHolder* H = reinterpret_cast<TcHolder*>(plans[0]->tc);
  TcBatch* B = H->cache;
  bool hit = B && B->prec == (int)prec && (int)B->plans.size() == count;
  for (int i = 0; hit && i < count; ++i) hit = B->plans[i] == plans[i] && B->serials[i] == plans[i]->serial;
  if (!hit) {
    tc_batch_destroy(H->cache);
    H->cache = nullptr;
    demag_status s = tc_batch_create(plans, count, prec, &H->cache);
    if (s != DEMAG_OK) return s;
    B = H->cache;
  }
  return tc_batch_run(B, m, phi, st);
}

// ---------------------------------------------------------------- analytic stray field

// Derivative factors of every axis and the three derivative stage programs
// (copies of the forward stage programs reading the derivative factors).
template <class F>
static demag_status prepare_field(demag_plan* P, TcState* S, cudaStream_t st) {
  if (S->field_ready) return DEMAG_OK;
  demag_status s = ensure_field_generators(P, st);
  if (s != DEMAG_OK) return s;
  const int M = P->M;
  for (int p = 0; p < 3; ++p) {
    const size_t bytes = (size_t)M * 2 * P->n[p] * S->ld[p] * S->elem;
    for (int h = 0; h < 2; ++h) {
      DEMAG_CUDA(P, cudaMalloc(&S->Bd[p][h], bytes));
      DEMAG_CUDA(P, cudaMemsetAsync(S->Bd[p][h], 0, bytes, st));
    }
    const long long total = (long long)M * 2 * P->n[p] * P->n[p];
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<F><<<grid_blocks(total), 256, 0, st>>>(
                     M, P->glen, p, P->n[p], S->ld[p], P->gend, P->scale, (typename F::T*)S->Bd[p][0],
                     (typename F::T*)S->Bd[p][1], nullptr, 0, 0));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  int t0[6];
  for (int st3 = 0; st3 < 3; ++st3) {
    TcGroup& G = S->dprog_host[st3];
    G = S->host_prog[kFwd1 + st3];
    if (!S->small[kFwd1 + st3]) {
      const int p = st3;  // stage s contracts axis s
      for (int h = 0; h < 2; ++h)
        if (!make_map(h ? &G.b_lo : &G.b_hi, S->Bd[p][h], S->elem, P->n[p], P->n[p], 2 * M, S->ld[p], G.bn))
          return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
    }
    S->small_dprog[st3] = S->small_prog[kFwd1 + st3];
    S->small_dprog[st3].gen = P->gend;
    S->small_dprog[st3].fac = nullptr;
    t0[2 * st3] = 0;
    t0[2 * st3 + 1] = G.ntiles;
  }
  DEMAG_CUDA(P, cudaMalloc(&S->dprog, sizeof(TcGroup) * 3));
  DEMAG_CUDA(P, cudaMalloc(&S->dtile0, sizeof(t0)));
  DEMAG_CUDA(P, cudaMemcpy(S->dprog, S->dprog_host, sizeof(TcGroup) * 3, cudaMemcpyHostToDevice));
  DEMAG_CUDA(P, cudaMemcpy(S->dtile0, t0, sizeof(t0), cudaMemcpyHostToDevice));
  S->field_ready = true;
  return DEMAG_OK;
}

template <class F>
static demag_status run_deriv(demag_plan* P, TcState* S, int st3, cudaStream_t st) {
  if (S->small[kFwd1 + st3]) return launch_small<F>(P, S->small_dprog[st3], st);
  return launch_groups<F>(P, S->dprog + st3, S->dtile0 + 2 * st3, 1, S->dprog_host[st3].ntiles, S->counter,
                          S->status, st);
}

// h_d[p] = -dphi/dxi_p.  The three chains share work: the stage-1 output feeds
// the directions 3 and 2, the stage-2 output direction 3, so eight stage
// launches give the three fields (three independent chains would take nine).
template <class F>
static demag_status field_chain(demag_plan* P, TcState* S, const float* m, float* hd, cudaStream_t st) {
  const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
  demag_status s = prepare_field<F>(P, S, st);
  if (s == DEMAG_OK) s = split_input<F>(P, S, m, 3, st);
  // direction 3: stages 1, 2 as for phi, derivative stage 3
  if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd1, st);
  if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd2, st);
  if (s == DEMAG_OK) s = run_deriv<F>(P, S, 2, st);
  if (s == DEMAG_OK) s = reduce_parts(P, S, S->groups_fwd, 1, -1.f, hd + 2 * N, st);
  // direction 2: derivative stage 2 on the stage-1 output, stage 3 as for phi
  if (s == DEMAG_OK) s = run_deriv<F>(P, S, 1, st);
  if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd3, st);
  if (s == DEMAG_OK) s = reduce_parts(P, S, S->groups_fwd, 1, -1.f, hd + N, st);
  // direction 1: derivative stage 1, stages 2 and 3 as for phi
  if (s == DEMAG_OK) s = run_deriv<F>(P, S, 0, st);
  if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd2, st);
  if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd3, st);
  if (s == DEMAG_OK) s = reduce_parts(P, S, S->groups_fwd, 1, -1.f, hd, st);
  return s;
}

demag_status tc_field(demag_plan* P, const float* m, float* hd, demag_precision prec, cudaStream_t st) {
  demag_status s = tc_prepare(P, prec, st);
  if (s != DEMAG_OK) return s;
  TcState* S = state(P, prec);
  return prec == DEMAG_TF32X3 ? field_chain<Tf32Form>(P, S, m, hd, st) : field_chain<Bf16Form>(P, S, m, hd, st);
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
