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
// block); a job is one output field (or one half of it, below) with a list of
// (A field, B matrix) pairs whose contractions it sums.  Several grids of
// different shapes therefore run a stage in one persistent launch.
//
// Even / odd halves.  On a uniform grid every 1D factor is Toeplitz with an
// even generator (E, Eq. f_anal) or an odd one (F), so with J the reversal of
// an axis J E J = E and J F J = -F (centro-symmetric and skew
// centro-symmetric).  Writing an axis of n cells (padded by one empty cell
// to n_e = 2h when n is odd) as x+_j = x_j + x_{n_e-1-j}, x-_j = x_j - x_{n_e-1-j},
// j < h, turns E into diag(E+, E-) and F into [[0, F-], [F+, 0]] with the
// h x h blocks
//     T+-[a][j] = T[a - j] +- T[a - (n_e - 1 - j)]
// (terms with |d| >= n vanish): y+ = E+ x+, y- = E- x- and y+ = F- x-,
// y- = F+ x+.  The input is folded once on every axis longer than 16 cells
// (fold_split_kernel), each mode product then contracts h instead of n
// entries (half the MMAs), and the node-sum reduction unfolds the potential
// (x_j = (x+ + x-)/2, x_{n_e-1-j} = (x+ - x-)/2).  In the split layout a folded
// axis has extent 2 hq (the odd half starts at hq = h rounded up to a 16-byte
// multiple); a job covers one output half, and a pair's contraction reads the
// input half given by its factor type.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc_ptx.cuh"

namespace demag {

constexpr int kBM = 128, kBN = 256;
constexpr int kRowBytes = 64;                      // one 64-byte swizzled row per k-block
constexpr int kMaxStages = 8;                      // operand ring depth: as many stages as fit (per launch)
constexpr int kTileA = kBM * kRowBytes;            // 8 KB
constexpr int kBarBytes = 1024;
// Epilogue warps: kEpiWarps / 4 warps share each TMEM lane quadrant and take
// its 32-column chunks in turn.  Four (one per quadrant) are faster than
// eight with two staging buffers each (256^3 stage 1: 1.22 against 1.48 ms):
// more stores in flight slow the output stream down.
#ifndef DEMAG_TC_EPI_WARPS
#define DEMAG_TC_EPI_WARPS 4
#endif
constexpr int kEpiWarps = DEMAG_TC_EPI_WARPS;
static_assert(kEpiWarps == 4 || kEpiWarps == 8, "4 or 8 epilogue warps");
constexpr int kEpiSlices = kEpiWarps / 4;          // warps per TMEM lane quadrant
constexpr int kOutBuf = 4096;                      // one 32 x 32 output chunk (2 BF16 planes or 1 FP32)
constexpr int kOutBufsPerWarp = 2;
constexpr int kOutStaging = kOutBufsPerWarp * kEpiWarps * kOutBuf;  // epilogue staging buffers
// dynamic shared memory: alignment slack, the operand stages (each A_hi, A_lo
// of 128 rows and B_hi, B_lo of the launch's widest N tile), staging, barriers
constexpr int kSmemFixed = 1024 + kOutStaging + kBarBytes;
constexpr int kSmemMax = 227 * 1024;
constexpr int kTcThreads = 64 + 32 * kEpiWarps;
constexpr int kRing = 4;                           // tile ids handed from the producer to the other roles
// Every pipeline wait gives up after the plan's wait limit (default 2 s,
// demag_set_wait_limit); the drains of the abort path always allow 2 s.
constexpr uint64_t kDrainNs = 2000000000ull;
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
  int pair0, npairs, out_field;
  int half;                            // output half (0 even, 1 odd; 0 on an axis not folded)
};

// One GEMM stage of one grid, in device memory (aligned as its tensor maps).
struct alignas(128) TcGroup {
  CUtensorMap a_hi, a_lo;              // 3D maps: (K, rows, field)
  CUtensorMap b_hi, b_lo;              // 4D maps: (K, a, half, matrix)
  CUtensorMap o_hi, o_lo;              // 5D output maps (inner, outer, a, half, field) when tma_out
  CUtensorMap w_hi, w_lo;              // the same with 128-row boxes (o_wide)
  const TcJob* jobs;
  const short2* pairs;                 // (A field, B matrix 2k + type)
  void* out_hi;                        // split: hi plane base; f32: float base
  void* out_lo;                        // split: lo plane base
  long long field_elems;               // elements per output field
  long long s_a;                       // output stride of the column index a
  int ldC, n_inner;                    // output row stride and row split (outer, inner)
  int rows, n_a, kblocks, bn, mode, tma_out;
  int o_wide;                          // one 128-row box per chunk from all epilogue warps (w_hi, w_lo);
                                       // a launch's groups are either all wide or none (shared staging)
  int hq;                              // folded axis: start of the odd half (K and output columns), else 0
  int pxor;                            // 1 when type 0 factors are the odd ones (derivative factors)
  int a_mn;                            // A read MN-major (BF16): maps (rows, K, field) with 64-row boxes
  float alpha;
  int njobs, m_tiles, n_tiles, ntiles;
};

// A launch's tiles are cut into segments, contiguous in launch order: each a
// block of jobs and row blocks of one group (tile order inside: row block,
// then job, then column tile), with field offsets for the A operand and the
// output (ring buffers), an optional dependency (a counter that must reach a
// value before the segment's operands are loaded) and an optional completion
// counter (each epilogue warp adds 1 after its stores of a tile are visible).
struct TcSeg {
  int group;                           // index into TcLaunch::groups
  int tile0;                           // first launch tile of the segment
  int job0, njobs;                     // jobs [job0, job0 + njobs) of the group
  int rb0, nrb;                        // row blocks [rb0, rb0 + nrb)
  int a_fofs, o_fofs;                  // added to every A field / output field
  int dep, dep_target;                 // wait for counters[dep] >= dep_target (dep < 0: none)
  int done;                            // completion counter (< 0: none)
  int order;                           // 0: row block outer, job, column tile; 1: job outer
};

struct TcLaunch {
  const TcGroup* groups;               // device array
  const TcSeg* segs;                   // device array, ascending tile0
  int nsegs, total_tiles;
  int nstages;                         // operand stages in the ring (<= kMaxStages)
  int btile;                           // bytes of one B plane tile: widest N tile x 64
  int stage_bytes;                     // 2 kTileA + 2 btile
  int* tile_counter;                   // zeroed before the launch
  int* counters;                       // dependency counters, zeroed before the launch (or NULL)
  int* status;
  unsigned long long wait_ns;          // limit of every pipeline wait
};

struct TileRef {
  int seg, g, j, mt, nt;
};

__device__ __forceinline__ TileRef tile_coords(const TcLaunch& L, int tile) {
  int lo = 0, hi = L.nsegs - 1;
  while (lo < hi) {  // last segment whose first tile <= tile
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&L.segs[mid].tile0) <= tile) lo = mid; else hi = mid - 1;
  }
  const TcSeg& S = L.segs[lo];
  const TcGroup& G = L.groups[S.group];
  int t = tile - S.tile0;
  TileRef r;
  r.seg = lo;
  r.g = S.group;
  r.nt = t % G.n_tiles;
  t /= G.n_tiles;
  if (S.order) {  // every row block of one job in turn
    r.mt = S.rb0 + t % S.nrb;
    r.j = S.job0 + t / S.nrb;
  } else {        // every job of one row block in turn (they share its A rows in L2)
    r.j = S.job0 + t % S.njobs;
    r.mt = S.rb0 + t / S.njobs;
  }
  return r;
}

// Count one epilogue warp's part of `count` finished tiles on completion
// counter `ctr`: their stores must be visible at GPU scope first.  TMA stores:
// all but the `keep` newest bulk groups of lane 0 (a later tile's) must be
// complete; direct stores: the warp's lanes are ordered before lane 0's release.
__device__ __forceinline__ void epi_signal(int* counters, int ctr, int count, bool tma, int keep, int lane) {
  __syncwarp();
  if (lane == 0) {
    if (tma) {
      ptx::bulk_wait_keep(keep);
      ptx::fence_proxy_async_global();
    }
    __threadfence();
    ptx::red_release_gpu_add(counters + ctr, count);
  }
  __syncwarp();
}

__device__ __forceinline__ void tc_fail(volatile int* abort, int* status) {
  *abort = 1;
  atomicExch(status, (int)DEMAG_ETIMEOUT);
}

template <class F>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(const __grid_constant__ TcLaunch L) {
  using T = typename F::T;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nst = L.nstages;
  const int stage_bytes = L.stage_bytes;
  // operand stages first, then the epilogue staging (both 1024-aligned), then
  // the barriers; staging placed first measured 4-9% slower in stages 1 and 2
  uint8_t* smem = base;
  uint8_t* ostage = base + nst * stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(ostage + kOutStaging);
  const int btile = L.btile;
  uint64_t* empty = full + kMaxStages;
  uint64_t* tfull = empty + kMaxStages;  // [2]
  uint64_t* tempty = tfull + 2;        // [2]
  uint64_t* drain = tempty + 2;        // [1]
  uint64_t* sfull = drain + 1;         // [kRing] a tile id is in the ring slot
  uint64_t* sempty = sfull + kRing;    // [kRing] the MMA thread and the 4 epilogue warps read it
  uint64_t* oready = sempty + kRing;   // [2] wide stores: every epilogue warp staged its rows
  uint64_t* ofree = oready + 2;        // [2] wide stores: the store that read the buffer has read it
  volatile int* ring = reinterpret_cast<volatile int*>(ofree + 2);  // [kRing]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(const_cast<int*>(ring) + kRing);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
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
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(&oready[b], kEpiWarps);
      ptx::mbar_init(&ofree[b], 1);
    }
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
  // producer: stages armed at least once, and the phase parity of their last
  // arming (an aborted launch waits for those loads to land before exiting)
  uint32_t armed = 0, armed_par = 0;

  if (warp == 0) {
    {
      // the whole warp runs the loop (converged); lane 0 issues the copies
      const bool leader = lane == 0;
      int s = 0;
      uint32_t ph = 0;
      int rs = 0;
      uint32_t rph = 0;
      int met_dep = -1, met_target = 0;  // last dependency seen satisfied (counters only grow)
      while (!*abort) {
        // take the next tile and hand its id to the MMA and epilogue roles
        if (!ptx::mbar_wait_warp(&sempty[rs], rph ^ 1, abort, L.wait_ns)) {
          if (leader) tc_fail(abort, L.status);
          break;
        }
        int tile = 0;
        if (leader) {
          tile = atomicAdd(L.tile_counter, 1);
          ring[rs] = tile < L.total_tiles ? tile : -1;
          ptx::mbar_arrive(&sfull[rs]);
        }
        tile = __shfl_sync(0xffffffffu, tile, 0);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile >= L.total_tiles) break;
        const TileRef tr = tile_coords(L, tile);
        const TcSeg& SG = L.segs[tr.seg];
        const TcGroup& G = L.groups[tr.g];
        const TcJob J = G.jobs[tr.j];
        const int mt = tr.mt, nt = tr.nt;
        if (SG.dep >= 0 && !(SG.dep == met_dep && SG.dep_target <= met_target)) {
          // the operands of this segment are written by earlier tiles of the launch
          const bool met = ptx::counter_wait(L.counters + SG.dep, SG.dep_target, abort, L.wait_ns);
          if (!__all_sync(0xffffffffu, met)) {
            if (leader) tc_fail(abort, L.status);
            break;
          }
          ptx::fence_proxy_async_global();  // their generic-proxy release before our TMA reads
          met_dep = SG.dep;
          met_target = SG.dep_target;
        }
        const uint32_t bytes = 2 * kTileA + 2 * (uint32_t)G.bn * kRowBytes;
        for (int pi = 0; pi < J.npairs && !*abort; ++pi) {
          short2 pr = G.pairs[J.pair0 + pi];
          pr.x = (short)(pr.x + SG.a_fofs);
          // input half read by this pair: the output half for an even factor,
          // the other one for an odd factor
          const int koff = ((J.half ^ (pr.y & 1) ^ G.pxor) & 1) * G.hq;
          for (int kb = 0; kb < G.kblocks; ++kb) {
            if (!ptx::mbar_wait_warp(&empty[s], ph ^ 1, abort, L.wait_ns)) {
              if (leader) tc_fail(abort, L.status);
              break;
            }
            uint8_t* st = smem + s * stage_bytes;
            armed |= 1u << s;
            armed_par = (armed_par & ~(1u << s)) | (ph << s);
            if (!leader) {
              if (++s == nst) { s = 0; ph ^= 1; }
              continue;
            }
            ptx::mbar_arrive_expect_tx(&full[s], bytes);
            if (F::kElem == 2 && G.a_mn) {
              // rows contiguous, K the outer coordinate: two 64-row boxes per plane
              const int kc = koff + kb * F::kBK;
              ptx::tma_load_3d(st, &G.a_hi, &full[s], mt * kBM, kc, pr.x);
              ptx::tma_load_3d(st + kTileA / 2, &G.a_hi, &full[s], mt * kBM + 64, kc, pr.x);
              ptx::tma_load_3d(st + kTileA, &G.a_lo, &full[s], mt * kBM, kc, pr.x);
              ptx::tma_load_3d(st + kTileA + kTileA / 2, &G.a_lo, &full[s], mt * kBM + 64, kc, pr.x);
            } else {
              ptx::tma_load_3d(st, &G.a_hi, &full[s], koff + kb * F::kBK, mt * kBM, pr.x);
              ptx::tma_load_3d(st + kTileA, &G.a_lo, &full[s], koff + kb * F::kBK, mt * kBM, pr.x);
            }
            ptx::tma_load_4d(st + 2 * kTileA, &G.b_hi, &full[s], kb * F::kBK, nt * G.bn, J.half, pr.y);
            ptx::tma_load_4d(st + 2 * kTileA + btile, &G.b_lo, &full[s], kb * F::kBK, nt * G.bn, J.half, pr.y);
            if (++s == nst) { s = 0; ph ^= 1; }
          }
        }
      }
    }
  } else if (warp == 1) {
    {
      // the whole warp runs the loop (converged); lane 0 issues the MMAs and commits
      const bool leader = lane == 0;
      int s = 0;
      uint32_t ph = 0, tph = 0;
      int buf = 0;
      int rs = 0;
      uint32_t rph = 0;
      while (!*abort) {
        if (!ptx::mbar_wait_warp(&sfull[rs], rph, abort, L.wait_ns)) {
          if (leader) tc_fail(abort, L.status);
          break;
        }
        const int tile = ring[rs];
        __syncwarp();
        if (leader) ptx::mbar_arrive(&sempty[rs]);
        if (++rs == kRing) { rs = 0; rph ^= 1; }
        if (tile < 0) break;
        const TileRef tr = tile_coords(L, tile);
        const TcGroup& G = L.groups[tr.g];
        const TcJob J = G.jobs[tr.j];
        // an MN-major A tile: 32 K rows of 128 bytes per 64-row box (atoms of 8
        // rows 1024 bytes apart), the second box kTileA / 2 further
        const bool amn = F::kElem == 2 && G.a_mn;
        const uint32_t idesc = ptx::instr_desc(F::kFormat, kBM, (uint32_t)G.bn) | (amn ? ptx::kInstrAMajorMN : 0u);
        const int kblocks = G.kblocks;
        if (!ptx::mbar_wait_warp(&tempty[buf], tph ^ 1, abort, L.wait_ns)) {
          if (leader) tc_fail(abort, L.status);
          break;
        }
        ptx::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(buf * kBN);
        uint32_t acc = 0;
        bool ok = true;
        for (int pi = 0; pi < J.npairs && ok; ++pi) {
          for (int kb = 0; kb < kblocks; ++kb) {
            if (!ptx::mbar_wait_warp(&full[s], ph, abort, L.wait_ns)) {
              if (leader) tc_fail(abort, L.status);
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t st = ptx::smem_u32(smem + s * stage_bytes);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint32_t off = kk * 32;  // one MMA consumes 32 bytes of K
              const uint64_t ah = amn ? ptx::smem_desc_mn128(st + kk * 2048, kTileA / 2, 1024)
                                      : ptx::smem_desc(st + off, kSBO, kSwizzle64);
              const uint64_t al = amn ? ptx::smem_desc_mn128(st + kTileA + kk * 2048, kTileA / 2, 1024)
                                      : ptx::smem_desc(st + kTileA + off, kSBO, kSwizzle64);
              const uint64_t bh = ptx::smem_desc(st + 2 * kTileA + off, kSBO, kSwizzle64);
              const uint64_t bl = ptx::smem_desc(st + 2 * kTileA + btile + off, kSBO, kSwizzle64);
              if (leader) {
                F::mma(d, ah, bh, idesc, acc);
                F::mma(d, ah, bl, idesc, 1u);
                F::mma(d, al, bh, idesc, 1u);
              }
              acc = 1u;
            }
            issued_mma = true;
            if (leader) ptx::mma_commit(&empty[s]);
            if (++s == nst) { s = 0; ph ^= 1; }
          }
        }
        if (!ok) break;
        if (leader) ptx::mma_commit(&tfull[buf]);
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
    // Finished tiles are counted on their completion counter in one release
    // per run of tiles of the same counter: when a tile of another counter
    // follows (after that tile's own stores are issued, so the earlier ones
    // have had a tile's time to land), or as soon as the warp would otherwise
    // wait for work.  A warp never waits while holding counts that a later
    // tile may depend on.
    int pend = -1;       // completion counter of the tiles not yet counted
    int pend_n = 0;      // how many
    bool pend_tma = false;
    while (!*abort) {
      if (pend >= 0 && !ptx::mbar_try_wait(&sfull[rs], rph)) {
        epi_signal(L.counters, pend, pend_n, pend_tma, 0, lane);
        pend = -1;
      }
      if (!ptx::mbar_wait(&sfull[rs], rph, abort, L.wait_ns)) {
        tc_fail(abort, L.status);
        break;
      }
      const int tile = ring[rs];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (tile < 0) break;
      const TileRef tr = tile_coords(L, tile);
      const TcSeg& SG = L.segs[tr.seg];
      const TcGroup& G = L.groups[tr.g];
      const int out_field = G.jobs[tr.j].out_field + SG.o_fofs;
      const int half = G.jobs[tr.j].half;
      const int mt = tr.mt, nt = tr.nt;
      if (pend >= 0 && !ptx::mbar_try_wait(&tfull[buf], tph)) {
        epi_signal(L.counters, pend, pend_n, pend_tma, 0, lane);
        pend = -1;
      }
      if (!ptx::mbar_wait(&tfull[buf], tph, abort, L.wait_ns)) {
        tc_fail(abort, L.status);
        break;
      }
      ptx::tc_fence_after();
      int commits = 0;  // bulk groups lane 0 commits for this tile
      const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * kBN);
      const int a0 = nt * G.bn;
      const int bn = G.bn;
      const int n_inner = G.n_inner;
      const int mode = G.mode;
      const float alpha = G.alpha;
      if (G.tma_out && G.o_wide) {
        // The tile's 128 rows lie in one `outer` (n_inner % 128 == 0): the four
        // warps stage each 32-column chunk together as [column][128 rows] and
        // one thread stores it as one box per plane (rows of 128 elements, a
        // quarter of the store requests of per-warp boxes).  Two staging
        // buffers in turn: `oready` (every warp staged its rows) and `ofree`
        // (the store that last read the buffer has read it), both bounded.
        const int r0 = mt * kBM;
        const int outer0 = r0 / n_inner, inner0 = r0 - outer0 * n_inner;
        const bool issuer = warp == 2 && lane == 0;
        bool ok = true;
        for (int c0 = 0; c0 < bn && ok; c0 += 32) {
          uint32_t r[32];
          ptx::tmem_ld32(taddr + (uint32_t)c0, r);
          ptx::tmem_ld_wait(r);
          const uint32_t b = chunk & 1u, par = (chunk >> 1) & 1u;
          ++chunk;
          uint8_t* sb = ostage + b * (4 * kOutBuf);
          if (!ptx::mbar_wait(&ofree[b], par ^ 1u, abort, L.wait_ns)) {
            tc_fail(abort, L.status);
            ok = false;
            break;
          }
          const int rr = quad * 32 + lane;
          if (mode == kOutSplit) {
            T* sh = reinterpret_cast<T*>(sb);
            T* sl = sh + 32 * kBM;
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              T hi, lo;
              F::split(__uint_as_float(r[jj]), hi, lo);
              sh[jj * kBM + rr] = hi;
              sl[jj * kBM + rr] = lo;
            }
          } else {
            float* sf = reinterpret_cast<float*>(sb);
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) sf[jj * kBM + rr] = alpha * __uint_as_float(r[jj]);
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&oready[b]);
          if (issuer) {
            if (!ptx::mbar_wait(&oready[b], par, abort, L.wait_ns)) {
              tc_fail(abort, L.status);
              ok = false;
            } else {
              ptx::tma_store_5d(&G.w_hi, sb, inner0, outer0, a0 + c0, half, out_field);
              if (mode == kOutSplit)
                ptx::tma_store_5d(&G.w_lo, sb + 32 * kBM * sizeof(T), inner0, outer0, a0 + c0, half, out_field);
              ptx::bulk_commit();
              ++commits;
              // the previous chunk's store has read the other buffer: free it
              ptx::bulk_wait_read<1>();
              if (chunk >= 2) ptx::mbar_arrive(&ofree[b ^ 1u]);
            }
          }
          __syncwarp();
        }
        if (!ok) break;
      } else if (G.tma_out) {
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
          ptx::tmem_ld_wait(r);
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
            // the map's column extent is the half's valid count: columns past
            // it (padding, or the other half) are not written
            ptx::tma_store_5d(&G.o_hi, sb, inner_w, outer_w, a0 + c0, half, out_field);
            if (mode == kOutSplit)
              ptx::tma_store_5d(&G.o_lo, sb + 32 * 32 * sizeof(T), inner_w, outer_w, a0 + c0, half, out_field);
            ptx::bulk_commit();
          }
          ++commits;
        }
      } else {
        const int row = mt * kBM + rloc;
        const bool valid = row < G.rows;
        const int outer = row / n_inner, inner = row - outer * n_inner;
        const long long s_a = G.s_a;
        const long long rbase = (long long)out_field * G.field_elems + (long long)outer * G.ldC + inner +
                                (long long)(half * G.hq) * s_a;
        const int acount = min(bn, G.n_a - a0);  // columns of this tile that exist (in its half)
        for (int c0 = 32 * slice; c0 < bn; c0 += 32 * kEpiSlices) {
          uint32_t r[32];
          ptx::tmem_ld32(taddr + (uint32_t)c0, r);
          ptx::tmem_ld_wait(r);
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
      if (pend >= 0 && pend != SG.done) {  // earlier tiles' stores: all but this tile's newest groups
        epi_signal(L.counters, pend, pend_n, pend_tma, G.tma_out ? commits : 0, lane);
        pend = -1;
      }
      // later tiles of the launch read what this tile wrote; a wide tile's stores
      // are all issued by warp 2, which counts them for every epilogue warp
      const int wgt = G.o_wide ? (warp == 2 ? kEpiWarps : 0) : 1;
      if (SG.done >= 0 && wgt) {
        if (pend < 0) {
          pend = SG.done;
          pend_n = 0;
          pend_tma = false;
        }
        pend_n += wgt;
        pend_tma = pend_tma || G.tma_out != 0;
      }
    }
    if (pend >= 0) epi_signal(L.counters, pend, pend_n, pend_tma, 0, lane);
    if (lane == 0) ptx::bulk_wait_all();  // staged stores finished before the block exits
  }

  // teardown: after an abort let in-flight MMAs and copies land (each wait
  // bounded by kDrainNs) before the shared memory and TMEM are released.  The
  // epilogue warps have waited for their bulk stores after their loop.
  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (*abort) {
    volatile int no_abort = 0;
    if (warp == 1 && lane == 0 && issued_mma) {  // every MMA issued so far
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, &no_abort, kDrainNs);
    }
    if (threadIdx.x == 0)  // the last loads into every stage: their phase completes when they land
      for (int st = 0; st < nst; ++st)
        if (armed & (1u << st)) ptx::mbar_wait(&full[st], (armed_par >> st) & 1u, &no_abort, kDrainNs);
    __syncthreads();
  }
  if (warp == 1) ptx::tmem_dealloc(tmem_base, 512);
}

// ---------------------------------------------------------------- fused mode-1 / mode-2 products
//
// On a grid whose axes are all folded, with h1, h2 <= 128 entries per half on
// the first two, the mode-1 and mode-2 products of a slab i3
// run in one persistent kernel and the mode-1 results never leave the SM.  A
// unit is (slab i3, node k, output half h1o of axis 1).  Its mode-1 products
// are formed transposed, the factor block being the A operand:
//     Y_q[a1][i2] = sum_j1 T1_{k,q}[h1o][a1][j1] X_q[i3][i2][off1 + j1],
// so the accumulator holds one a1 per TMEM lane with i2 along the columns;
// split into BF16 hi / lo, every 32 columns of it are one K-major k-block of
// the A operand of the mode-2 product
//     Z[a1][a2] = sum_i2 Y[a1][i2] T2_{k,type}[h2o][a2][i2],
// handed over in shared memory (never written to the workspace).  Z is stored
// as [field][i3][a2][a1] (a1 contiguous, U_k field 2k, V_k field 2k + 1),
// which the mode-3 stage reads MN-major (TcGroup::a_mn).  Halves that are not
// multiples of 32: the contractions run over ceil(h / 32) k-blocks (factor
// columns past h read as zeros, Y columns past h2 are zeroed), the tiles are
// n2 = h2 rounded up to 16 wide, and the Z stores are clipped to the h1 x h2
// valid entries of each half by their tensor map.  Per unit six chunks
// (component q, input half hh of axis 2), each a mode-1 tile (128 x h2) and
// its mode-2 product, in an order that completes one target before the next:
//     c     0  1  2  3  4  5
//     q     0  1  0  1  2  2
//     hh    0  1  1  0  0  1
//   target U0 U0 U1 U1 V0 V1  (U_k = Y_1 x2 E + Y_2 x2 F, V_k = Y_3 x2 E; the
// index is the output half h2o = hh for E, hh ^ 1 for F).  Roles (10 warps):
//   warp 0      TMA producer, in the MMA's order: per chunk the mode-1
//               k-blocks (A: factor block, 128 rows; B: h2 rows of X) and the
//               mode-2 k-blocks (B: factor block of axis 2),
//   warp 1      MMA issuer: the mode-1 tile into the mode-1 accumulator, then
//               its mode-2 product (A from the Y slots) into the target's,
//   warps 2..5  mode-1 epilogue: accumulator -> hi / lo -> Y slots (a ring of
//               k-blocks in shared memory, handed to the MMA by mbarriers),
//   warps 6..9  mode-2 epilogue: accumulator -> hi / lo -> Z (TMA stores).
// Within a CTA these hand-offs serialise (a mode-1 tile, its conversion, the
// mode-2 product, the next tile), so a CTA takes half of an SM: 256 TMEM
// columns (one 128-column accumulator per mode) and ~106 KB of shared memory,
// and two CTAs share each SM's tensor core, one filling the other's gaps.
// The roles that issue copies and MMAs run their loops on the whole warp and
// issue from lane 0 (single-lane loops issued the MMAs measurably slower).
// Every wait is bounded as in tc_gemm_kernel, with the same abort path.
constexpr int kS12Threads = 320;
constexpr int kS12Ring = 4;                       // operand slots, one k-block of one operand (hi + lo)
constexpr int kS12RingSlot = 2 * kTileA;
constexpr int kS12Y = 2;                          // Y slots, one k-block of Y each (hi and lo)
constexpr int kS12YSlot = 2 * kTileA;
constexpr int kS12Plane = 32 * 32 * 2;            // one 32 x 32 BF16 plane: the staging of a mode-2 epilogue warp
constexpr int kS12Staging = 4 * kS12Plane;
constexpr int kS12Smem = 1024 + kS12Ring * kS12RingSlot + kS12Y * kS12YSlot + kS12Staging + kBarBytes;
constexpr int kS12Tmem = 256;                     // columns: mode-1 accumulator at 0, mode-2 at 128
static_assert(2 * (kS12Smem + 1024) <= 228 * 1024, "two fused CTAs per SM");

struct S12Launch {
  CUtensorMap t1_hi, t1_lo;            // axis-1 factor blocks, 128-row boxes (mode-1 A)
  CUtensorMap x_hi, x_lo;              // split input, n2-row boxes (mode-1 B)
  CUtensorMap t2_hi, t2_lo;            // axis-2 factor blocks, n2-row boxes (mode-2 B)
  CUtensorMap z_hi, z_lo;              // Z as (a1 < h1, half, a2 < h2, half, field), 32 x 32 store boxes
  int M, x2, x3;                       // nodes, extents of axes 2 (= 2 hq2) and 3
  int h1, h2;                          // valid entries per half of axes 1, 2
  int hq1, hq2;                        // start of the odd half of axes 1, 2 (h rounded up to 8)
  int n2;                              // tile width of both products: h2 rounded up to 16
  int kb1, kb2;                        // k-blocks of the two contractions (ceil(h1 / 32), ceil(h2 / 32))
  int pxor1, pxor2;                    // 1 when axis 1 / 2 carries derivative factors (dE odd, dF even)
  int units;                           // ext3 * M * 2 (batched: all items' units)
  int* unit_counter;                   // zeroed before the launch
  int* status;
  unsigned long long wait_ns;
  // batched launch (several grids, units numbered item after item): the
  // geometry and maps above come from items[i], the unit counter, status and
  // wait limit from the launch; null for a single grid
  const S12Launch* items;
  const int* unit0;                    // first unit of each item, [count + 1]
  int count;
};

// The launch that a unit of item `it` belongs to.
template <bool BATCH>
__device__ __forceinline__ const S12Launch& s12_item(const S12Launch& L, int it) {
  if constexpr (BATCH) return L.items[it];
  else return L;
}

// Chunk c of a unit: the field of X read by its mode-1 tile, the factor types
// along axes 1 and 2, the input half hh of axis 2, and whether it starts /
// completes its mode-2 target.  Forward: the table above.  Adjoint (the
// transposed chain, one input field y): Ya = y x1 F (chunks 0, 1), Yb = y x1 E
// (chunks 2-5, computed twice), targets Za = Ya x2 E (chunks 0, 1), Zb = Yb x2 F
// (2, 3), Zc = Yb x2 E (4, 5), one chunk each, in chunk order.
struct S12Chunk {
  int xf, type1, hh, type2;
  bool first, last;
};

template <bool ADJ>
__device__ __forceinline__ S12Chunk s12_chunk(int c) {
  S12Chunk r;
  if (!ADJ) {
    const int q = c < 4 ? (c & 1) : 2;
    r.xf = q;
    r.type1 = q == 0 ? 1 : 0;  // F along axis 1 for component 1
    r.hh = c < 4 ? (((c >> 1) ^ c) & 1) : (c & 1);
    r.type2 = q == 1 ? 1 : 0;  // F along axis 2 for component 2
    r.first = c < 4 ? (c & 1) == 0 : true;
    r.last = c < 4 ? (c & 1) == 1 : true;
  } else {
    r.xf = 0;
    r.type1 = c < 2 ? 1 : 0;
    r.hh = c & 1;
    r.type2 = (c >> 1) == 1 ? 1 : 0;
    r.first = r.last = true;
  }
  return r;
}

// Mode-2 target j of a unit (in the order they complete): its field within the
// node (forward U, V; adjoint Za, Zb, Zc) and its output half of axis 2.
template <bool ADJ>
__device__ __forceinline__ void s12_target(int j, int pxor2, int& zf, int& h2o) {
  zf = j >> 1;
  if (!ADJ) {
    h2o = (j & 1) ^ pxor2;
  } else {
    const S12Chunk ch = s12_chunk<true>(j);
    h2o = ch.hh ^ ch.type2 ^ pxor2;
  }
}

// hi / lo BF16 of two consecutive values, packed (the first in the low half)
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

template <bool ADJ, bool BATCH>
__global__ void __launch_bounds__(kS12Threads, 2) tc_s12_kernel(const __grid_constant__ S12Launch L) {
  constexpr int kTargets = ADJ ? 6 : 4;  // mode-2 targets per unit
  constexpr int kZf = ADJ ? 3 : 2;       // Z fields per node
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* slots = base;
  uint8_t* yslots = slots + kS12Ring * kS12RingSlot;
  uint8_t* ostage = yslots + kS12Y * kS12YSlot;
  uint64_t* full = reinterpret_cast<uint64_t*>(ostage + kS12Staging);
  uint64_t* empty = full + kS12Ring;
  uint64_t* d1full = empty + kS12Ring;     // the mode-1 accumulator
  uint64_t* d1empty = d1full + 1;
  uint64_t* yfull = d1empty + 1;           // [kS12Y]
  uint64_t* yempty = yfull + kS12Y;
  uint64_t* d2full = yempty + kS12Y;       // the mode-2 accumulator
  uint64_t* d2empty = d2full + 1;
  uint64_t* sfull = d2empty + 1;           // [kRing] unit ids
  uint64_t* sempty = sfull + kRing;
  uint64_t* drain = sempty + kRing;
  volatile int* ring = reinterpret_cast<volatile int*>(drain + 1);  // [kRing] unit within its item
  volatile int* ritem = ring + kRing;                                // [kRing] item of the unit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(const_cast<int*>(ritem) + kRing);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kS12Ring; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kS12Y; ++i) {
      ptx::mbar_init(&yfull[i], 4);
      ptx::mbar_init(&yempty[i], 1);
    }
    ptx::mbar_init(d1full, 1);
    ptx::mbar_init(d1empty, 4);
    ptx::mbar_init(d2full, 1);
    ptx::mbar_init(d2empty, 4);
    for (int i = 0; i < kRing; ++i) {
      ptx::mbar_init(&sfull[i], 1);
      ptx::mbar_init(&sempty[i], 9);
    }
    ptx::mbar_init(drain, 1);
    *abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(tmem_slot, kS12Tmem);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  bool issued_mma = false;
  uint32_t armed = 0, armed_par = 0;

  if (warp == 0) {
    // the whole warp runs the loop; lane 0 issues the copies
    const bool leader = lane == 0;
    int s = 0;
    uint32_t ph = 0;
    int rs = 0;
    uint32_t rph = 0;
    int cur = 0;  // item of the last unit taken (batched launch)
    bool ok = true;
    // next operand slot (its previous contents consumed), or null after an abort
    auto take_slot = [&]() -> uint8_t* {
      if (!ptx::mbar_wait_warp(&empty[s], ph ^ 1, abort, L.wait_ns)) {
        if (leader) tc_fail(abort, L.status);
        ok = false;
        return nullptr;
      }
      armed |= 1u << s;
      armed_par = (armed_par & ~(1u << s)) | (ph << s);
      return slots + s * kS12RingSlot;
    };
    auto next_slot = [&]() {
      if (++s == kS12Ring) {
        s = 0;
        ph ^= 1;
      }
    };
    while (ok && !*abort) {
      if (!ptx::mbar_wait_warp(&sempty[rs], rph ^ 1, abort, L.wait_ns)) {
        if (leader) tc_fail(abort, L.status);
        break;
      }
      int u = 0, it = 0;
      if (leader) {
        u = atomicAdd(L.unit_counter, 1);
        if (u >= L.units) {
          u = -1;
        } else if (BATCH) {  // this CTA's units only grow: the item cursor only advances
          while (cur + 1 < L.count && u >= L.unit0[cur + 1]) ++cur;
          it = cur;
          u -= L.unit0[cur];
        }
        ring[rs] = u;
        ritem[rs] = it;
        ptx::mbar_arrive(&sfull[rs]);
      }
      u = __shfl_sync(0xffffffffu, u, 0);
      it = __shfl_sync(0xffffffffu, it, 0);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (u < 0) break;
      const S12Launch& G = s12_item<BATCH>(L, it);
      const int h1o = u & 1, k = (u >> 1) % G.M, i3 = (u >> 1) / G.M;
      for (int c = 0; c < 6 && ok; ++c) {
        const S12Chunk ch = s12_chunk<ADJ>(c);
        const int q = ch.xf, hh = ch.hh, type1 = ch.type1;
        // mode 1: factor block of (k, type) and h2 rows of X_q (input half hh of axis 2)
        const int off1 = ((h1o ^ type1 ^ G.pxor1) & 1) * G.hq1;  // input half of axis 1
        const int row = i3 * G.x2 + hh * G.hq2;
        for (int kb = 0; kb < G.kb1 && ok; ++kb) {
          uint8_t* a = take_slot();
          if (!a) break;
          if (leader) {
            ptx::mbar_arrive_expect_tx(&full[s], 2 * kTileA);
            ptx::tma_load_4d(a, &G.t1_hi, &full[s], kb * 32, 0, h1o, 2 * k + type1);
            ptx::tma_load_4d(a + kTileA, &G.t1_lo, &full[s], kb * 32, 0, h1o, 2 * k + type1);
          }
          next_slot();
          uint8_t* b = take_slot();
          if (!b) break;
          if (leader) {
            ptx::mbar_arrive_expect_tx(&full[s], 2 * G.n2 * kRowBytes);
            ptx::tma_load_3d(b, &G.x_hi, &full[s], off1 + kb * 32, row, q);
            ptx::tma_load_3d(b + kTileA, &G.x_lo, &full[s], off1 + kb * 32, row, q);
          }
          next_slot();
        }
        // mode 2: factor block of (k, type, h2o)
        const int type2 = ch.type2;
        for (int kb = 0; kb < G.kb2 && ok; ++kb) {
          uint8_t* b = take_slot();
          if (!b) break;
          if (leader) {
            ptx::mbar_arrive_expect_tx(&full[s], 2 * G.n2 * kRowBytes);
            // the block of the output half h2o = hh ^ type (^ 1 for derivative factors)
            ptx::tma_load_4d(b, &G.t2_hi, &full[s], kb * 32, 0, hh ^ type2 ^ G.pxor2, 2 * k + type2);
            ptx::tma_load_4d(b + kTileA, &G.t2_lo, &full[s], kb * 32, 0, hh ^ type2 ^ G.pxor2, 2 * k + type2);
          }
          next_slot();
        }
      }
    }
  } else if (warp == 1) {
    // the whole warp runs the loop; lane 0 issues the MMAs and commits
    const bool leader = lane == 0;
    int s = 0;
    uint32_t ph = 0;
    int rs = 0;
    uint32_t rph = 0;
    uint32_t t = 0, yc = 0, g = 0;  // mode-1 tiles, Y k-blocks consumed, mode-2 targets completed
    bool ok = true;
    const uint32_t d1 = tmem_base, d2 = tmem_base + 128;
    // the next operand slot once its loads have landed (index in `idx`)
    auto take_full = [&](int& idx) -> uint32_t {
      if (!ptx::mbar_wait_warp(&full[s], ph, abort, L.wait_ns)) {
        if (leader) tc_fail(abort, L.status);
        ok = false;
        return 0;
      }
      ptx::tc_fence_after();
      idx = s;
      const uint32_t a = ptx::smem_u32(slots + s * kS12RingSlot);
      if (++s == kS12Ring) {
        s = 0;
        ph ^= 1;
      }
      return a;
    };
    while (ok && !*abort) {
      if (!ptx::mbar_wait_warp(&sfull[rs], rph, abort, L.wait_ns)) {
        if (leader) tc_fail(abort, L.status);
        break;
      }
      const int u = ring[rs], it = ritem[rs];
      __syncwarp();
      if (leader) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (u < 0) break;
      const S12Launch& G = s12_item<BATCH>(L, it);
      const int kb1 = G.kb1, kb2 = G.kb2;
      const uint32_t idesc = ptx::instr_desc(1, kBM, (uint32_t)G.n2);
      for (int c = 0; c < 6 && ok; ++c) {
        // mode 1 into the mode-1 accumulator, once the previous tile is read out
        if (!ptx::mbar_wait_warp(d1empty, (t & 1) ^ 1, abort, L.wait_ns)) {
          if (leader) tc_fail(abort, L.status);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int kb = 0; kb < kb1 && ok; ++kb) {
          int ia = 0, ib = 0;
          const uint32_t sa = take_full(ia);
          const uint32_t sb = ok ? take_full(ib) : 0;
          if (!ok) break;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t ah = ptx::smem_desc(sa + off, kSBO, kSwizzle64);
            const uint64_t al = ptx::smem_desc(sa + kTileA + off, kSBO, kSwizzle64);
            const uint64_t bh = ptx::smem_desc(sb + off, kSBO, kSwizzle64);
            const uint64_t bl = ptx::smem_desc(sb + kTileA + off, kSBO, kSwizzle64);
            if (leader) {
              Bf16Form::mma(d1, ah, bh, idesc, (kb | kk) ? 1u : 0u);
              Bf16Form::mma(d1, ah, bl, idesc, 1u);
              Bf16Form::mma(d1, al, bh, idesc, 1u);
            }
          }
          issued_mma = true;
          if (leader) {
            ptx::mma_commit(&empty[ia]);
            ptx::mma_commit(&empty[ib]);
          }
        }
        if (!ok) break;
        if (leader) ptx::mma_commit(d1full);
        ++t;
        // mode 2 into the target's accumulator
        const S12Chunk ch = s12_chunk<ADJ>(c);
        const bool first = ch.first, last = ch.last;
        if (first) {
          if (!ptx::mbar_wait_warp(d2empty, (g & 1) ^ 1, abort, L.wait_ns)) {
            if (leader) tc_fail(abort, L.status);
            ok = false;
            break;
          }
          ptx::tc_fence_after();
        }
        for (int kb = 0; kb < kb2 && ok; ++kb) {
          const uint32_t ys = yc % kS12Y;
          if (!ptx::mbar_wait_warp(&yfull[ys], (yc / kS12Y) & 1, abort, L.wait_ns)) {
            if (leader) tc_fail(abort, L.status);
            ok = false;
            break;
          }
          int ib = 0;
          const uint32_t sb = take_full(ib);
          if (!ok) break;
          const uint32_t ya = ptx::smem_u32(yslots + ys * kS12YSlot);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            const uint32_t off = kk * 32;
            const uint64_t ah = ptx::smem_desc(ya + off, kSBO, kSwizzle64);
            const uint64_t al = ptx::smem_desc(ya + kTileA + off, kSBO, kSwizzle64);
            const uint64_t bh = ptx::smem_desc(sb + off, kSBO, kSwizzle64);
            const uint64_t bl = ptx::smem_desc(sb + kTileA + off, kSBO, kSwizzle64);
            if (leader) {
              Bf16Form::mma(d2, ah, bh, idesc, (first && kb == 0 && kk == 0) ? 0u : 1u);
              Bf16Form::mma(d2, ah, bl, idesc, 1u);
              Bf16Form::mma(d2, al, bh, idesc, 1u);
            }
          }
          issued_mma = true;
          ++yc;
          // each k-block's slots are released as soon as its MMAs complete
          // (batching two k-blocks per commit measured 4% slower here: with two
          // Y slots the mode-1 epilogue then waits for both)
          if (leader) {
            ptx::mma_commit(&empty[ib]);
            ptx::mma_commit(&yempty[ys]);
          }
        }
        if (!ok) break;
        if (last) {
          if (leader) ptx::mma_commit(d2full);
          ++g;
        }
      }
    }
  } else if (warp < 6) {
    // mode-1 epilogue: row a1 = quad * 32 + lane of the accumulator; each
    // 32-column block becomes one k-block of Y: 64-byte rows in the 64-byte
    // swizzle of the TMA (16-byte chunk c of row r at c ^ ((r >> 1) & 3))
    const int quad = warp & 3;
    const int r = quad * 32 + lane;
    const uint32_t rowoff = (uint32_t)r * 64, sw = (uint32_t)(r >> 1) & 3u;
    const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16);
    int rs = 0;
    uint32_t rph = 0;
    uint32_t t = 0, yc = 0;
    bool ok = true;
    while (ok && !*abort) {
      if (!ptx::mbar_wait(&sfull[rs], rph, abort, L.wait_ns)) {
        tc_fail(abort, L.status);
        break;
      }
      const int u = ring[rs], it = ritem[rs];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (u < 0) break;
      const S12Launch& G = s12_item<BATCH>(L, it);
      const int kb2 = G.kb2, h2 = G.h2;
      for (int c = 0; c < 6 && ok; ++c) {
        if (!ptx::mbar_wait(d1full, t & 1, abort, L.wait_ns)) {
          tc_fail(abort, L.status);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        for (int kb = 0; kb < kb2; ++kb) {
          uint32_t v[32];
          ptx::tmem_ld32(taddr + (uint32_t)(kb * 32), v);
          const uint32_t ys = yc % kS12Y;
          if (!ptx::mbar_wait(&yempty[ys], ((yc / kS12Y) & 1) ^ 1, abort, L.wait_ns)) {
            ptx::tmem_ld_wait(v);
            tc_fail(abort, L.status);
            ok = false;
            break;
          }
          ptx::tmem_ld_wait(v);
          if (kb + 1 == kb2) {  // the accumulator is read: the next mode-1 tile may start
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(d1empty);
            // columns i2 >= h2: rows of the next half or never written; zero
            // them, so that Y holds only finite entries (their factor columns
            // read as zeros)
            const int lim = h2 - kb * 32;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (j >= lim) v[j] = 0u;
          }
          uint8_t* slot = yslots + ys * kS12YSlot;
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            uint32_t hw[4], lw[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              split_pair(__uint_as_float(v[cc * 8 + 2 * e]), __uint_as_float(v[cc * 8 + 2 * e + 1]), hw[e], lw[e]);
            const uint32_t o = rowoff + (((uint32_t)cc ^ sw) << 4);
            *reinterpret_cast<uint4*>(slot + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
            *reinterpret_cast<uint4*>(slot + kTileA + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) ptx::mbar_arrive(&yfull[ys]);
          ++yc;
        }
        ++t;
      }
    }
  } else {
    // mode-2 epilogue: rows a1 of the unit's output half, columns a2; each
    // 32 x 32 chunk staged as [a2][a1], plane by plane, one box each.
    // Targets in the order they complete: U0, U1, V0, V1 (their output halves
    // swapped when axis 2 carries derivative factors).
    const int quad = warp & 3;
    uint8_t* stg = ostage + (warp - 6) * kS12Plane;
    const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + 128;
    int rs = 0;
    uint32_t rph = 0;
    uint32_t g = 0;
    bool ok = true;
    while (ok && !*abort) {
      if (!ptx::mbar_wait(&sfull[rs], rph, abort, L.wait_ns)) {
        tc_fail(abort, L.status);
        break;
      }
      const int u = ring[rs], it = ritem[rs];
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&sempty[rs]);
      if (++rs == kRing) { rs = 0; rph ^= 1; }
      if (u < 0) break;
      const S12Launch& G = s12_item<BATCH>(L, it);
      const int h1o = u & 1, k = (u >> 1) % G.M, i3 = (u >> 1) / G.M;
      const bool valid = quad * 32 < G.h1;  // rows past h1 are zero and not stored
      for (int j = 0; j < kTargets && ok; ++j) {
        if (!ptx::mbar_wait(d2full, g & 1, abort, L.wait_ns)) {
          tc_fail(abort, L.status);
          ok = false;
          break;
        }
        ptx::tc_fence_after();
        int tf, h2o;
        s12_target<ADJ>(j, G.pxor2, tf, h2o);
        const int zf = i3 + G.x3 * (kZf * k + tf);
        for (int c0 = 0; c0 < G.h2; c0 += 32) {
          uint32_t v[32];
          ptx::tmem_ld32(taddr + (uint32_t)c0, v);
          ptx::tmem_ld_wait(v);
          if (!valid) continue;
          __nv_bfloat16* sp = reinterpret_cast<__nv_bfloat16*>(stg);
#pragma unroll
          for (int pl = 0; pl < 2; ++pl) {
            // the previous store has read the buffer
            if (lane == 0) ptx::bulk_wait_read<0>();
            __syncwarp();
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              __nv_bfloat16 hi, lo;
              Bf16Form::split(__uint_as_float(v[jj]), hi, lo);
              sp[jj * 32 + lane] = pl ? lo : hi;
            }
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
              // (a1 in the half, output half of axis 1, a2 in the target's half, its half, field)
              ptx::tma_store_5d(pl ? &G.z_lo : &G.z_hi, stg, quad * 32, h1o, c0, h2o, zf);
              ptx::bulk_commit();
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(d2empty);
        ++g;
      }
    }
    if (lane == 0) ptx::bulk_wait_all();
  }

  __syncwarp();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  if (*abort) {
    volatile int no_abort = 0;
    if (warp == 1 && lane == 0 && issued_mma) {
      ptx::mma_commit(drain);
      ptx::mbar_wait(drain, 0, &no_abort, kDrainNs);
    }
    if (threadIdx.x == 0)
      for (int st = 0; st < kS12Ring; ++st)
        if (armed & (1u << st)) ptx::mbar_wait(&full[st], (armed_par >> st) & 1u, &no_abort, kDrainNs);
    __syncthreads();
  }
  if (warp == 1) ptx::tmem_dealloc(tmem_base, kS12Tmem);
}

// ---------------------------------------------------------------- operand preparation

// Element-wise kernels over several grids in one launch: item i covers the
// flat range [begin_i, begin_{i+1}) of the launch's index space; a thread's
// indices only grow, so it finds its item by advancing from the last one.
constexpr int kMaxItems = 128;

// Geometry of one grid in the split layout: per axis the cell count n, the
// valid entries per half h, the start of the odd half hq and the extent ext
// (2 hq on a folded axis; n, h = n, hq = 0 otherwise).
struct AxisGeo {
  int n[3], h[3], hq[3], ext[3];
};

struct FoldItem {
  const float* x;      // [fields][n3][n2][n1] FP32
  void* hi;            // [fields][ext3][ext2][ld1] planes
  void* lo;
  long long begin;     // first row of this item in the launch's row space
  AxisGeo g;
  int ld1;
};

struct FoldList {
  int count;
  long long total;     // rows (field, j3, j2) over all items
  FoldItem it[kMaxItems];
};

// Orbit counts per axis: a folded axis has hq positions per half (the last
// hq - h of them padding), an axis not folded n.
__device__ __forceinline__ int orbit_count(const AxisGeo& g, int p) { return g.hq[p] ? g.hq[p] : g.n[p]; }

// Fold every folded axis of [fields][n3][n2][n1] FP32 tensors into even / odd
// halves (x+- = x_j +- x_{n_e-1-j}, the padding cell of an odd axis being 0)
// and split the result into hi / lo planes.  A block takes one orbit row
// (field, j3, j2) at a time; its threads take the orbits j1 of the row: each
// reads the up to 8 cells (j or n_e-1-j on each folded axis) once and writes
// the up to 8 folded entries (even or odd half on each folded axis), so reads
// and writes are coalesced along i1.
template <class F>
__global__ void __launch_bounds__(128) fold_split_kernel(const __grid_constant__ FoldList L) {
  using T = typename F::T;
  int item = 0;
  for (long long r = blockIdx.x; r < L.total; r += gridDim.x) {
    while (item + 1 < L.count && r >= L.it[item + 1].begin) ++item;
    const FoldItem& S = L.it[item];
    const AxisGeo& g = S.g;
    const int c1 = orbit_count(g, 0), c2 = orbit_count(g, 1), c3 = orbit_count(g, 2);
    int e = (int)(r - S.begin);
    const int j2 = e % c2;
    e /= c2;
    const int j3 = e % c3;
    const int q = e / c3;
    const int f1 = g.hq[0] ? 1 : 0, f2 = g.hq[1] ? 1 : 0, f3 = g.hq[2] ? 1 : 0;
    const bool live = j2 < g.h[1] && j3 < g.h[2];
    // source rows for (e3, e2) and destination rows for (s3, s2), index e2 + 2 e3
    const float* src[4];
    long long dst[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int b2 = k & 1, b3 = k >> 1;
      const int m2 = b2 ? 2 * g.h[1] - 1 - j2 : j2, m3 = b3 ? 2 * g.h[2] - 1 - j3 : j3;
      const bool ok = live && b2 <= f2 && b3 <= f3 && m2 < g.n[1] && m3 < g.n[2];
      src[k] = ok ? S.x + (((long long)q * g.n[2] + m3) * g.n[1] + m2) * g.n[0] : nullptr;
      dst[k] = (b2 <= f2 && b3 <= f3)
                   ? (((long long)q * g.ext[2] + b3 * g.hq[2] + j3) * g.ext[1] + b2 * g.hq[1] + j2) * S.ld1
                   : -1;
    }
    if (F::kElem == 2 && f1 && (g.n[0] & 3) == 0 && (reinterpret_cast<uintptr_t>(S.x) & 7) == 0) {
      // n1 a multiple of 4 (h1 even): two neighbouring orbits per thread, both
      // valid or both padding, their cells and their mirror cells each an
      // aligned float2, the outputs a BF16 pair
      const int fl[3] = {f1, f2, f3};
      for (int j1 = 2 * threadIdx.x; j1 < c1; j1 += 2 * blockDim.x) {
        const bool l1 = j1 < g.h[0];
        float v[2][8];
#pragma unroll
        for (int row = 0; row < 4; ++row) {
          float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
          if (src[row] && l1) {
            a = __ldg(reinterpret_cast<const float2*>(src[row] + j1));
            b = __ldg(reinterpret_cast<const float2*>(src[row] + 2 * g.h[0] - 2 - j1));
          }
          v[0][2 * row] = a.x;      // orbit j1: cell j1, mirror 2h - 1 - j1
          v[0][2 * row + 1] = b.y;
          v[1][2 * row] = a.y;      // orbit j1 + 1
          v[1][2 * row + 1] = b.x;
        }
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            if (!fl[p]) continue;
            const int bit = 1 << p;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (!(k & bit)) {
                const float a = v[o][k], b = v[o][k | bit];
                v[o][k] = a + b;
                v[o][k | bit] = a - b;
              }
          }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int b1 = k & 1, row = k >> 1;
          if (dst[row] < 0) continue;
          const long long o = dst[row] + b1 * g.hq[0] + j1;
          uint32_t hw, lw;
          split_pair(v[0][k], v[1][k], hw, lw);
          *reinterpret_cast<uint32_t*>(reinterpret_cast<T*>(S.hi) + o) = hw;
          *reinterpret_cast<uint32_t*>(reinterpret_cast<T*>(S.lo) + o) = lw;
        }
      }
      continue;
    }
    for (int j1 = threadIdx.x; j1 < c1; j1 += blockDim.x) {
      const bool l1 = j1 < g.h[0];
      const int m1[2] = {j1, 2 * g.h[0] - 1 - j1};
      float v[8];  // [e3][e2][e1], then [s3][s2][s1] after the butterflies
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int b1 = k & 1, row = k >> 1;
        float x = 0.f;
        if (src[row] && l1 && b1 <= f1 && m1[b1] < g.n[0]) x = __ldg(src[row] + m1[b1]);
        v[k] = x;
      }
      const int fl[3] = {f1, f2, f3};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        if (!fl[p]) continue;
        const int bit = 1 << p;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (!(k & bit)) {
            const float a = v[k], b = v[k | bit];
            v[k] = a + b;
            v[k | bit] = a - b;
          }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int b1 = k & 1, row = k >> 1;
        if (dst[row] < 0 || b1 > f1) continue;
        const long long o = dst[row] + b1 * g.hq[0] + j1;
        T h, l;
        F::split(v[k], h, l);
        reinterpret_cast<T*>(S.hi)[o] = h;
        reinterpret_cast<T*>(S.lo)[o] = l;
      }
    }
  }
}

// Dense factors of one axis, hi/lo: on an axis not folded the Toeplitz
// matrix [M][2][n][ldB] (or the non-uniform grid's full matrix); on a folded
// axis the blocks [M][2][2 halves][h][ldB] of the header (even half: T+ for
// an even factor, T- for an odd one; odd half: the other sign).  The third
// axis carries the scale c s omega_k.  pxor = 1 swaps the parity of the two
// factor types (the derivative factors of the stray field: dE odd, dF even).
template <class F>
__global__ void tc_factor_kernel(int M, int glen, int axis, int n, int h, int halves, int ldB, int pxor,
                                 const double* gen, const double* scale, typename F::T* hi, typename F::T* lo,
                                 const double* fac, size_t tgroup, size_t toff) {
  const long long total = (long long)M * 2 * halves * h * h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(i % h);
    long long t = i / h;
    const int ii = (int)(t % h);
    t /= h;
    const int half = (int)(t % halves);
    const int kt = (int)(t / halves);  // k*2 + type
    const double* row = gen + ((long long)kt * 3 + axis) * glen + (n - 1);  // row[d] = T[d], |d| < n
    double v;
    if (fac) {
      v = fac[(size_t)kt * tgroup + toff + (size_t)ii * n + jj];  // non-uniform grid: never folded
    } else if (halves == 1) {
      v = row[ii - jj];
    } else {
      const int jm = 2 * h - 1 - jj;
      const int dm = ii - jm;
      const double t2 = (dm > -n && dm < n) ? row[dm] : 0.0;
      const bool even = ((kt & 1) ^ pxor) == 0;
      v = ((half == 0) == even) ? row[ii - jj] + t2 : row[ii - jj] - t2;
    }
    if (axis == 2) v *= scale[kt / 2];
    typename F::T hv, lv;
    F::split((float)v, hv, lv);
    const long long o = (((long long)kt * halves + half) * h + ii) * ldB + jj;
    hi[o] = hv;
    lo[o] = lv;
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

struct UnfoldItem {
  const float* part;   // [nout][groups][ext3][ext2][ext1] partial fields
  float* out;          // [nout][n3][n2][n1]
  long long begin;     // first row of this item in the launch's row space
  AxisGeo g;
  int groups;
  float alpha;         // includes 1/2 per folded axis
};

struct UnfoldList {
  int count;
  long long total;     // rows (output field, j3, j2) over all items
  UnfoldItem it[kMaxItems];
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

// out[q] = alpha * unfold(sum_g part[q][g]): the node-sum partial fields are
// summed (compensated), then every folded axis is unfolded
// (x_j = x+ + x-, x_{n_e-1-j} = x+ - x-, the 1/2 in alpha).  A block takes one
// orbit row (field, j3, j2) of valid entries (j < h) at a time, its threads
// the orbits j1 of the row; the loads of up to kUnfoldBatch partial fields
// are issued together before they are summed.
constexpr int kUnfoldBatch = 4;

__global__ void __launch_bounds__(128, 6) unfold_reduce_kernel(const __grid_constant__ UnfoldList L) {
  int item = 0;
  for (long long r = blockIdx.x; r < L.total; r += gridDim.x) {
    while (item + 1 < L.count && r >= L.it[item + 1].begin) ++item;
    const UnfoldItem& R = L.it[item];
    const AxisGeo& g = R.g;
    int e = (int)(r - R.begin);
    const int j2 = e % g.h[1];
    e /= g.h[1];
    const int j3 = e % g.h[2];
    const int q = e / g.h[2];
    const int f1 = g.hq[0] ? 1 : 0, f2 = g.hq[1] ? 1 : 0, f3 = g.hq[2] ? 1 : 0;
    const long long fe = (long long)g.ext[0] * g.ext[1] * g.ext[2];
    const float* base = R.part + (long long)q * R.groups * fe;
    // source rows for (s3, s2) and destination rows for (e3, e2), index b2 + 2 b3
    const float* src[4];
    float* dst[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int b2 = k & 1, b3 = k >> 1;
      const bool on = b2 <= f2 && b3 <= f3;
      src[k] = on ? base + ((long long)(b3 * g.hq[2] + j3) * g.ext[1] + b2 * g.hq[1] + j2) * g.ext[0] : nullptr;
      const int m2 = b2 ? 2 * g.h[1] - 1 - j2 : j2, m3 = b3 ? 2 * g.h[2] - 1 - j3 : j3;
      dst[k] = (on && m2 < g.n[1] && m3 < g.n[2])
                   ? R.out + (((long long)q * g.n[2] + m3) * g.n[1] + m2) * g.n[0]
                   : nullptr;
    }
    if (f1 && (g.n[0] & 3) == 0 && (reinterpret_cast<uintptr_t>(R.out) & 7) == 0) {
      // n1 a multiple of 4 (h1 even): two neighbouring orbits per thread, each
      // partial read and each output (and its mirror) written as a float2
      const int fl[3] = {f1, f2, f3};
      for (int j1 = 2 * threadIdx.x; j1 < g.h[0]; j1 += 2 * blockDim.x) {
        Csum a[2][8];
        for (int gi = 0; gi < R.groups; ++gi) {
          float2 x[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int b1 = k & 1, row = k >> 1;
            x[k] = src[row] ? __ldg(reinterpret_cast<const float2*>(src[row] + gi * fe + b1 * g.hq[0] + j1))
                            : make_float2(0.f, 0.f);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            a[0][k].add(x[k].x);
            a[1][k].add(x[k].y);
          }
        }
        float v[2][8];
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int k = 0; k < 8; ++k) v[o][k] = a[o][k].value();
#pragma unroll
        for (int o = 0; o < 2; ++o)
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            if (!fl[p]) continue;
            const int bit = 1 << p;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (!(k & bit)) {
                const float u = v[o][k], w = v[o][k | bit];
                v[o][k] = u + w;
                v[o][k | bit] = u - w;
              }
          }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int b1 = k & 1, row = k >> 1;
          if (!dst[row]) continue;
          if (b1 == 0)  // cells j1, j1 + 1
            *reinterpret_cast<float2*>(dst[row] + j1) = make_float2(R.alpha * v[0][k], R.alpha * v[1][k]);
          else          // mirror cells 2h - 2 - j1 (of orbit j1 + 1) and 2h - 1 - j1 (of orbit j1)
            *reinterpret_cast<float2*>(dst[row] + 2 * g.h[0] - 2 - j1) =
                make_float2(R.alpha * v[1][k], R.alpha * v[0][k]);
        }
      }
      continue;
    }
    for (int j1 = threadIdx.x; j1 < g.h[0]; j1 += blockDim.x) {
      Csum a[8];
      for (int g0 = 0; g0 < R.groups; g0 += kUnfoldBatch) {
        const int ng = min(kUnfoldBatch, R.groups - g0);
        float x[8][kUnfoldBatch];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int b1 = k & 1, row = k >> 1;
#pragma unroll
          for (int gi = 0; gi < kUnfoldBatch; ++gi)
            x[k][gi] = (src[row] && b1 <= f1 && gi < ng)
                           ? __ldg(src[row] + (g0 + gi) * fe + b1 * g.hq[0] + j1)
                           : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
          for (int gi = 0; gi < kUnfoldBatch; ++gi)
            if (gi < ng) a[k].add(x[k][gi]);
      }
      float v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = a[k].value();
      const int fl[3] = {f1, f2, f3};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        if (!fl[p]) continue;
        const int bit = 1 << p;
#pragma unroll
        for (int k = 0; k < 8; ++k)
          if (!(k & bit)) {
            const float u = v[k], w = v[k | bit];
            v[k] = u + w;
            v[k | bit] = u - w;
          }
      }
      const int m1[2] = {j1, 2 * g.h[0] - 1 - j1};
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int b1 = k & 1, row = k >> 1;
        if (!dst[row] || b1 > f1 || m1[b1] >= g.n[0]) continue;
        dst[row][m1[b1]] = R.alpha * v[k];
      }
    }
  }
}

// Plans with no folded axis (non-uniform grids, grids whose axes all have at
// most kSmallAxis cells) use flat element-wise kernels instead: the row-wise
// ones would give each thread too few elements of a long unfolded row.

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

// One block of rows of one job of a stage (the block's threads all run the
// shared-memory rounds; rows past the stage's count only skip the arithmetic).
template <class F>
__device__ __forceinline__ void small_stage_block(const SmallStage& S, int job, int rowblock, float* sB) {
  using T = typename F::T;
  const TcJob J = S.jobs[job];
  const int n = S.n;
  const int row = rowblock * blockDim.x + threadIdx.x;
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

template <class F>
__global__ void __launch_bounds__(256) small_stage_kernel(const __grid_constant__ SmallStage S) {
  __shared__ float sB[kSmallChunk * kSmallAxis * kSmallAxis];
  small_stage_block<F>(S, blockIdx.y, blockIdx.x, sB);
}

// The thin last stages of several grids in one launch (batched applications):
// blockIdx.y runs over the jobs of all items, blockIdx.x over row blocks up to
// the largest item's; blocks past their item's rows leave at once.
constexpr int kMaxSmallItems = 32;
struct SmallBatch {
  SmallStage it[kMaxSmallItems];
  int job0[kMaxSmallItems + 1];  // first job of each item
  int count;
  int rowblocks;                 // of the largest item
};

template <class F>
__global__ void __launch_bounds__(256) small_batch_kernel(const __grid_constant__ SmallBatch B) {
  __shared__ float sB[kSmallChunk * kSmallAxis * kSmallAxis];
  int i = 0;
  while (i + 1 < B.count && (int)blockIdx.y >= B.job0[i + 1]) ++i;
  const SmallStage& S = B.it[i];
  if ((long long)blockIdx.x * blockDim.x >= S.rows) return;  // uniform over the block
  small_stage_block<F>(S, (int)blockIdx.y - B.job0[i], blockIdx.x, sB);
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

// 4D map over the factor blocks of one axis [2M][halves][h][ldB]:
// (K, a, half, matrix), box (64 bytes, box1, 1, 1), 64B swizzle.  Columns and
// rows past h read as zeros.
static bool make_bmap(CUtensorMap* m, void* base, int elem_bytes, uint64_t h, uint64_t halves, uint64_t mats,
                      uint64_t ldB, uint32_t box1) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[4] = {h, h, halves, mats};
  cuuint64_t strides[3] = {ldB * elem_bytes, ldB * h * elem_bytes, ldB * h * halves * elem_bytes};
  cuuint32_t box[4] = {(cuuint32_t)(kRowBytes / elem_bytes), box1, 1, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, 4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 5D map over an output field set: (inner, outer, a, half, field) with the
// given strides in elements, the column index a limited to the na valid
// columns of a half (the odd half starts hq columns after the even one);
// box (box_inner, 1, 32, 1, 1) = one epilogue warp's 32 rows (or the four
// warps' 128 rows) x 32 output columns, no swizzle.
static bool make_out_map(CUtensorMap* m, void* base, int elem_bytes, uint64_t inner, uint64_t outer, uint64_t na,
                         uint64_t halves, uint64_t hq, uint64_t fields, uint64_t ld, uint64_t s_a,
                         uint64_t field_elems, uint32_t box_inner = 32) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[5] = {inner, outer, na, halves, fields};
  const uint64_t s_half = (halves > 1 ? hq : na) * s_a;
  cuuint64_t strides[4] = {ld * elem_bytes, s_a * elem_bytes, s_half * elem_bytes, field_elems * elem_bytes};
  cuuint32_t box[5] = {box_inner, 1, 32, 1, 1};
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  const CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = enc(m, dt, 5, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 3D BF16 map with explicit strides, box and swizzle (the fused application's
// Z fields and its operand maps of other box shapes).
static bool make_map3(CUtensorMap* m, void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1_elems,
                      uint64_t s2_elems, uint32_t b0, uint32_t b1, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {s1_elems * 2, s2_elems * 2};
  cuuint32_t box[3] = {b0, b1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Stage programs of a plan: forward stages 0-2, adjoint stages 3-5, and the
// mode-3 stages of the fused forward and adjoint applications (A = Z read
// MN-major).
enum { kFwd1 = 0, kFwd2, kFwd3, kAdj1, kAdj2, kAdj3, kFwd3Z, kAdj3Z, kPrograms };
constexpr int kChain = kFwd3Z;  // programs of the three-stage chains

// axis contracted by stage program p
static int prog_axis(int p) { return p >= kChain ? 2 : p % 3; }

// Per-plan, per-form tensor-core state.
struct TcState {
  int elem;               // bytes per element (2 BF16, 4 TF32)
  AxisGeo geo;            // split layout per axis (folded into halves or not)
  int halves[3];          // 2 on a folded axis, else 1
  int ld[3];              // padded row lengths of the extents (16-byte multiples)
  int ldB[3];             // padded row length of the factor blocks
  int bn[3];              // N tile width per axis
  void* B[3][2];          // per axis: hi / lo factors [M][2][halves][h][ldB]
  void* X[2];             // split input: [3][ext3 ext2][ld1]
  void* buf1[2];          // [3M][ext1 ext3][ld2]
  void* buf2[2];          // [3M][ext2 ext1][ld3]
  int* status;
  int* counter;           // dynamic tile counter of the running launch
  float* part;            // split node-sum partial fields
  int pp3;                // (A, B) pairs per accumulator in the node-sum stage
  int part_fields;        // partial fields allocated
  int groups_fwd, groups_adj;  // partial fields used by the forward / adjoint node sum
  int tma[3];             // stage epilogue stores through TMA
  int wide[3];            // ... one 128-row box per chunk (n_inner % 128 == 0)
  // stage programs: the group descriptors (device) and their job / pair tables
  TcGroup* prog;          // device [kPrograms]
  TcJob* jobs;            // device, all programs
  short2* pairs;          // device, all programs
  TcSeg* seg;             // device [kPrograms]: one whole-program segment each
  TcSeg host_seg[kPrograms];
  int nst[kPrograms];     // operand stages of each program's launches (0: as many as fit)
  TcGroup host_prog[kPrograms];
  bool small[kPrograms];          // program runs on CUDA cores (axis of at most kSmallAxis cells)
  SmallStage small_prog[kPrograms];
  // fused forward application (tc_s12_kernel, then kFwd3Z): built where the
  // grid allows it (BF16x3, every axis folded, h1 and h2 at most 128); the Z
  // fields live in buf1
  bool fused;
  int sched;              // forward schedule (1 fused, 0 chain): the tuner's choice, else sched0
  int sched0;             // untuned forward schedule: fused on grids of at least 2^20 split cells
  S12Launch s12;
  S12Launch s12a;         // the adjoint's fused launch (Z with 3M fields)
  // analytic stray field: the forward stage programs with the derivative
  // factors of their axis (built on first use)
  bool field_ready;
  void* Bd[3][2];                 // per axis: hi / lo derivative factors [M][2][n][ld]
  TcGroup dprog_host[4];          // stages 1-3 with derivative factors; 3: the fused schedule's
                                  // mode-3 stage (Z, MN-major) with derivative factors
  TcGroup* dprog;                 // device [4]
  TcSeg* dseg;                    // device [4]
  SmallStage small_dprog[3];
  S12Launch s12d[2];              // fused launches with derivative factors along axis 1 / axis 2
  size_t bytes;
};

// The forward stages of several plans as one launch (every stage of every
// grid, later stages of a grid waiting for its earlier ones); owned by a
// plan's cache or by a captured graph.
struct TcBatch {
  std::vector<demag_plan*> plans;
  std::vector<unsigned long long> serials;  // with the pointers, the cache key
  int prec = -1;
  TcGroup* groups = nullptr;           // device [3][count]
  TcSeg* segs = nullptr;               // device [nsegs]
  int nsegs = 0, total = 0;
  int* ctr = nullptr;                  // device [1 + 2 count]: tile counter, then stage-done counters
  int nctr = 0;
  int maxbn = 16;                      // widest N tile of all groups
  std::vector<char> fused;             // per plan: the fused schedule (part of the cache key)
  S12Launch* s12items = nullptr;       // device [s12count]: the fused grids' mode-1/mode-2 launches
  int* s12unit0 = nullptr;             // device [s12count + 1]: first unit of each
  int s12count = 0, s12units = 0;
  SmallBatch small;                    // thin last stages run on CUDA cores after the persistent launch
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

// Split layout of a plan's grid for elements of `elem` bytes: every axis of a
// uniform grid longer than kSmallAxis cells is folded into even / odd halves.
struct TcGeo {
  AxisGeo g;
  int halves[3], ld[3], ldB[3];
};

static TcGeo tc_geometry(const demag_plan* P, int elem) {
  const int al = 16 / elem;
  TcGeo G;
  for (int p = 0; p < 3; ++p) {
    const int n = P->n[p];
    const bool fold = !P->nonuniform && n > kSmallAxis;
    G.g.n[p] = n;
    G.g.h[p] = fold ? (n + 1) / 2 : n;
    G.g.hq[p] = fold ? round_up(G.g.h[p], al) : 0;
    G.g.ext[p] = fold ? 2 * G.g.hq[p] : n;
    G.halves[p] = fold ? 2 : 1;
    G.ld[p] = round_up(G.g.ext[p], al);
    G.ldB[p] = round_up(G.g.h[p], al);
  }
  return G;
}

size_t tc_workspace_bytes(const demag_plan* P, demag_precision prec) {
  const size_t e = prec == DEMAG_TF32X3 ? 4 : 2;
  const TcGeo G = tc_geometry(P, (int)e);
  const size_t x1 = G.g.ext[0], x2 = G.g.ext[1], x3 = G.g.ext[2];
  size_t b = 0;
  for (int p = 0; p < 3; ++p) b += 2 * (size_t)P->M * 2 * G.halves[p] * G.g.h[p] * G.ldB[p] * e;
  b += 2 * 3 * x3 * x2 * G.ld[0] * e;
  b += 2 * 3 * (size_t)P->M * x1 * x3 * G.ld[1] * e;
  b += 2 * 3 * (size_t)P->M * x2 * x1 * G.ld[2] * e;
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
  cudaFree(S->seg);
  for (int p = 0; p < 3; ++p)
    for (int h = 0; h < 2; ++h) cudaFree(S->Bd[p][h]);
  cudaFree(S->dprog);
  cudaFree(S->dseg);
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

// blocks of a row-wise launch: one row per block, at most 16 blocks per SM
static int row_blocks(long long rows, int per_sm = 16) {
  const long long cap = 152LL * per_sm;
  return (int)(rows > cap ? cap : (rows < 1 ? 1 : rows));
}

static TcJob job(int pair0, int npairs, int out_field, int half) {
  TcJob j;
  j.pair0 = pair0;
  j.npairs = npairs;
  j.out_field = out_field;
  j.half = half;
  return j;
}

// matrix index of (node k, type) in the per-axis factor maps
static short mat(int k, int type) { return (short)(2 * k + type); }

// Build the six stage programs of a plan (host descriptors, job and pair tables).
struct ProgramBuild {
  std::vector<TcJob> jobs;
  std::vector<short2> pairs;
  int job0[kChain], pair0[kChain];
};

// The segment covering every tile of group `group`, starting at launch tile tile0.
static TcSeg whole_seg(const TcGroup& G, int group, int tile0) {
  TcSeg q;
  memset(&q, 0, sizeof(q));
  q.group = group;
  q.tile0 = tile0;
  q.job0 = 0;
  q.njobs = G.njobs;
  q.rb0 = 0;
  q.nrb = G.m_tiles;
  q.dep = -1;
  q.done = -1;
  return q;
}

static void set_stage(TcGroup& G, const CUtensorMap& ahi, const CUtensorMap& alo, const CUtensorMap& bhi,
                      const CUtensorMap& blo, int rows, int n_a, int K, int bk, int bn, void* out_hi, void* out_lo,
                      long long field_elems, long long s_a, int ldC, int n_inner, int mode, float alpha, int hq) {
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
  G.hq = hq;
  G.pxor = 0;
  G.m_tiles = (rows + kBM - 1) / kBM;
  G.n_tiles = (n_a + bn - 1) / bn;
}

static demag_status build_programs(demag_plan* P, TcState* S, const CUtensorMap (&mapX)[2],
                                   const CUtensorMap (&map1)[2], const CUtensorMap (&map2)[2],
                                   const CUtensorMap (&mapB)[3][2], const CUtensorMap (&out1)[2],
                                   const CUtensorMap (&out2)[2], const CUtensorMap& out3,
                                   const CUtensorMap (&wout1)[2], const CUtensorMap (&wout2)[2],
                                   const CUtensorMap& wout3, const CUtensorMap (&zA)[2],
                                   const CUtensorMap (&zA3)[2], int bk, cudaStream_t st) {
  const AxisGeo& g = S->geo;
  const int M = P->M;
  const int x1 = g.ext[0], x2 = g.ext[1], x3 = g.ext[2];
  const long long Nx = (long long)x1 * x2 * x3;
  ProgramBuild b;
  auto begin = [&](int prog) {
    b.job0[prog] = (int)b.jobs.size();
    b.pair0[prog] = (int)b.pairs.size();
  };
  // one job per output half, all reading the last npairs pairs pushed
  auto add_job = [&](int prog, int npairs, int out_field) {
    const int p0 = (int)b.pairs.size() - b.pair0[prog] - npairs;
    for (int hf = 0; hf < S->halves[prog_axis(prog)]; ++hf) b.jobs.push_back(job(p0, npairs, out_field, hf));
  };
  auto add_job_at = [&](int prog, int p0, int npairs, int out_field) {
    for (int hf = 0; hf < S->halves[prog_axis(prog)]; ++hf) b.jobs.push_back(job(p0, npairs, out_field, hf));
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
  for (int gi = 0; gi < S->groups_fwd; ++gi) {
    const int p0 = gi * S->pp3;
    const int np = (2 * M - p0) < S->pp3 ? (2 * M - p0) : S->pp3;
    add_job_at(kFwd3, p0, np, gi);
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
      add_job_at(kAdj3, base + p0, np, q * S->groups_adj + gi);
    }
  }
  const int job_end = (int)b.jobs.size();

  const long long f1 = (long long)x1 * x3 * S->ld[1], f2 = (long long)x2 * x1 * S->ld[2];
  TcGroup* H = S->host_prog;
  memset(H, 0, sizeof(S->host_prog));
  set_stage(H[kFwd1], mapX[0], mapX[1], mapB[0][0], mapB[0][1], x3 * x2, g.h[0], g.h[0], bk, S->bn[0], S->buf1[0],
            S->buf1[1], f1, (long long)x3 * S->ld[1], S->ld[1], x2, kOutSplit, 1.f, g.hq[0]);
  set_stage(H[kFwd2], map1[0], map1[1], mapB[1][0], mapB[1][1], x1 * x3, g.h[1], g.h[1], bk, S->bn[1], S->buf2[0],
            S->buf2[1], f2, (long long)x1 * S->ld[2], S->ld[2], x3, kOutSplit, 1.f, g.hq[1]);
  set_stage(H[kFwd3], map2[0], map2[1], mapB[2][0], mapB[2][1], x2 * x1, g.h[2], g.h[2], bk, S->bn[2], S->part,
            nullptr, Nx, (long long)x2 * x1, x1, x1, kOutF32, 1.f, g.hq[2]);
  H[kAdj1] = H[kFwd1];
  H[kAdj2] = H[kFwd2];
  H[kAdj3] = H[kFwd3];
  for (int p = 0; p < kChain; ++p) {
    const int stage = p % 3;
    if (S->tma[stage]) {
      H[p].tma_out = 1;
      H[p].o_wide = 0;  // per-warp boxes by default; the tuner may pick wide ones where S->wide
      if (stage == 0) { H[p].o_hi = out1[0]; H[p].o_lo = out1[1]; H[p].w_hi = wout1[0]; H[p].w_lo = wout1[1]; }
      if (stage == 1) { H[p].o_hi = out2[0]; H[p].o_lo = out2[1]; H[p].w_hi = wout2[0]; H[p].w_lo = wout2[1]; }
      if (stage == 2) { H[p].o_hi = out3; H[p].w_hi = wout3; }
    }
  }
  // job and pair tables
  DEMAG_CUDA(P, cudaMalloc(&S->jobs, sizeof(TcJob) * b.jobs.size()));
  DEMAG_CUDA(P, cudaMalloc(&S->pairs, sizeof(short2) * b.pairs.size()));
  DEMAG_CUDA(P, cudaMemcpy(S->jobs, b.jobs.data(), sizeof(TcJob) * b.jobs.size(), cudaMemcpyHostToDevice));
  DEMAG_CUDA(P, cudaMemcpy(S->pairs, b.pairs.data(), sizeof(short2) * b.pairs.size(), cudaMemcpyHostToDevice));
  for (int p = 0; p < kChain; ++p) {
    const int jend = p + 1 < kChain ? b.job0[p + 1] : job_end;
    H[p].jobs = S->jobs + b.job0[p];
    H[p].pairs = S->pairs + b.pair0[p];
    H[p].njobs = jend - b.job0[p];
    H[p].ntiles = H[p].njobs * H[p].m_tiles * H[p].n_tiles;
  }
  // the fused application's mode-3 stage: the forward mode-3 program with Z
  // ([field][i3][a2][a1]) as its A operand, read MN-major; the same rows
  // (a2, a1), pairs and output
  H[kFwd3Z] = H[kFwd3];
  H[kAdj3Z] = H[kAdj3];
  if (S->fused) {
    H[kFwd3Z].a_hi = zA[0];
    H[kFwd3Z].a_lo = zA[1];
    H[kFwd3Z].a_mn = 1;
    H[kAdj3Z].a_hi = zA3[0];  // the adjoint's Z: 3M fields
    H[kAdj3Z].a_lo = zA3[1];
    H[kAdj3Z].a_mn = 1;
  }
  // stages along an axis of at most kSmallAxis cells (never folded) run on CUDA cores
  {
    const void* in_hi[3] = {S->X[0], S->buf1[0], S->buf2[0]};
    const void* in_lo[3] = {S->X[1], S->buf1[1], S->buf2[1]};
    const long long rows_of[3] = {(long long)x3 * x2, (long long)x1 * x3, (long long)x2 * x1};
    for (int p = 0; p < kPrograms; ++p) {
      const int stage = prog_axis(p);
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
  for (int p = 0; p < kPrograms; ++p) S->host_seg[p] = whole_seg(H[p], 0, 0);
  DEMAG_CUDA(P, cudaMalloc(&S->seg, sizeof(S->host_seg)));
  DEMAG_CUDA(P, cudaMemcpy(S->seg, S->host_seg, sizeof(S->host_seg), cudaMemcpyHostToDevice));
  (void)st;
  return DEMAG_OK;
}

template <class F>
static demag_status prepare_form(demag_plan* P, TcState* S, cudaStream_t st) {
  const int M = P->M;
  for (int p = 0; p < 3; ++p) {
    const int h = S->geo.h[p];
    long long total = (long long)M * 2 * S->halves[p] * h * h;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<F><<<grid_blocks(total), 256, 0, st>>>(
                     M, P->glen, p, P->n[p], h, S->halves[p], S->ldB[p], 0, P->gen64, P->scale,
                     (typename F::T*)S->B[p][0], (typename F::T*)S->B[p][1], P->fac64, P->tgroup, P->toff[p]));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  static unsigned long long attr = 0;  // devices whose kernel attribute is set
  int dev = 0;
  DEMAG_CUDA(P, cudaGetDevice(&dev));
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr & bit)) {
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_gemm_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_s12_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kS12Smem));
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_s12_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kS12Smem));
    DEMAG_CUDA(P, cudaFuncSetAttribute(tc_s12_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kS12Smem));
    attr |= bit;
  }
  return DEMAG_OK;
}

template <class F>
static demag_status run_program(demag_plan* P, TcState* S, int prog, cudaStream_t st);
static demag_status run_s12(demag_plan* P, TcState* S, const S12Launch& base, cudaStream_t st, bool adj = false);

// Point stage program `prog` at output-column tile width bn (device copy included).
static demag_status set_tile_width(demag_plan* P, TcState* S, int prog, int bn) {
  TcGroup& G = S->host_prog[prog];
  const int axis = prog_axis(prog);
  const int M = P->M;
  for (int h = 0; h < 2; ++h)
    if (!make_bmap(h ? &G.b_lo : &G.b_hi, S->B[axis][h], S->elem, S->geo.h[axis], S->halves[axis], 2 * M,
                   S->ldB[axis], bn))
      return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  G.bn = bn;
  G.n_tiles = (G.n_a + bn - 1) / bn;
  G.ntiles = G.njobs * G.m_tiles * G.n_tiles;
  DEMAG_CUDA(P, cudaMemcpy(S->prog + prog, &G, sizeof(TcGroup), cudaMemcpyHostToDevice));
  return DEMAG_OK;
}

// Point stage program `prog` at tile order `order` (device copy included).
static demag_status set_tile_order(demag_plan* P, TcState* S, int prog, int order) {
  S->host_seg[prog].order = order;
  DEMAG_CUDA(P, cudaMemcpy(S->seg + prog, &S->host_seg[prog], sizeof(TcSeg), cudaMemcpyHostToDevice));
  return DEMAG_OK;
}

// Tuned entry kinds of the tensor-core programs, per form (BF16x3, TF32x3):
// N tile width 1 / 2, operand stages 3 / 4, tile order 5 / 6, store boxes
// 7 / 8 (per warp or one 128-row box per chunk); key = (stage program,
// default value, 0).
static int tune_kind(const TcState* S, int knob) { return 1 + 2 * knob + (S->elem == 2 ? 0 : 1); }

static const demag_plan::Tuned* find_tuned(const demag_plan* P, int kind, int prog) {
  for (const demag_plan::Tuned& t : P->tuned)
    if (t.kind == kind && t.key[0] == prog) return &t;
  return nullptr;
}

static demag_status set_knob(demag_plan* P, TcState* S, int prog, int knob, int v) {
  if (knob == 0) return set_tile_width(P, S, prog, v);
  if (knob == 1) {
    S->nst[prog] = v;
    return DEMAG_OK;
  }
  if (knob == 2) return set_tile_order(P, S, prog, v);
  // store boxes: wide ones only where the stage has them
  TcGroup& G = S->host_prog[prog];
  G.o_wide = (v && S->wide[prog_axis(prog)]) ? 1 : 0;
  DEMAG_CUDA(P, cudaMemcpy(S->prog + prog, &G, sizeof(TcGroup), cudaMemcpyHostToDevice));
  return DEMAG_OK;
}

// Tuned entry kind of the forward schedule (BF16x3): 1 fused, 0 chain; key (0, 1, 0).
constexpr int kTuneSchedule = 9;

// Apply tuned entries already in the plan (a loaded cache) to its programs.
static demag_status apply_tuned(demag_plan* P, TcState* S) {
  if (S->fused)
    for (const demag_plan::Tuned& t : P->tuned)
      if (t.kind == kTuneSchedule && (t.value == 0 || t.value == 1)) S->sched = t.value;
  for (int prog = 0; prog < kPrograms; ++prog) {
    if (S->small[prog] || (prog >= kChain && !S->fused)) continue;
    for (int knob = 0; knob < 4; ++knob) {
      const demag_plan::Tuned* t = find_tuned(P, tune_kind(S, knob), prog);
      if (!t) continue;
      if (knob == 0 && !(t->value >= 16 && t->value <= kBN && t->value % 16 == 0)) continue;
      demag_status s = set_knob(P, S, prog, knob, t->value);
      if (s != DEMAG_OK) return s;
    }
  }
  return DEMAG_OK;
}

// Autotuning of every stage program (one warm-up and three timed launches per
// candidate, operands as they are in the workspace), one knob after the other,
// each kept at its fastest value: the output-column tile width (the default:
// 256, or the column count rounded up to 16; 128 and 64 below it), the number
// of operand stages (as many as fit, 4, 3, 2), the tile order (every job of a
// row block in turn, or every row block of a job) and, where a 128-row block
// lies in one outer index, the store boxes (per warp, or one 128-row box per
// chunk from all four epilogue warps).  None of them changes the arithmetic of
// an output element.
template <class F>
static demag_status tune_programs(demag_plan* P, TcState* S, cudaStream_t st) {
  cudaEvent_t e0, e1;
  DEMAG_CUDA(P, cudaEventCreate(&e0));
  DEMAG_CUDA(P, cudaEventCreate(&e1));
  demag_status s = DEMAG_OK;
  // the stage launches of one forward application (operand split and node-sum
  // reduction are the same for both schedules and not timed)
  auto time_sched = [&](int fused, float* ms) -> demag_status {
    auto once = [&]() -> demag_status {
      if (fused) {
        demag_status r = run_s12(P, S, S->s12, st);
        return r == DEMAG_OK ? run_program<F>(P, S, kFwd3Z, st) : r;
      }
      demag_status r = DEMAG_OK;
      for (int prog = kFwd1; prog <= kFwd3 && r == DEMAG_OK; ++prog) r = run_program<F>(P, S, prog, st);
      return r;
    };
    demag_status r = once();
    if (r != DEMAG_OK) return r;
    DEMAG_CUDA(P, cudaEventRecord(e0, st));
    for (int i = 0; i < 3 && r == DEMAG_OK; ++i) r = once();
    DEMAG_CUDA(P, cudaEventRecord(e1, st));
    DEMAG_CUDA(P, cudaEventSynchronize(e1));
    if (r != DEMAG_OK) return r;
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= 3.f;
    return DEMAG_OK;
  };
  auto time_prog = [&](int prog, float* ms) -> demag_status {
    demag_status r = run_program<F>(P, S, prog, st);
    if (r != DEMAG_OK) return r;
    DEMAG_CUDA(P, cudaEventRecord(e0, st));
    for (int i = 0; i < 3 && r == DEMAG_OK; ++i) r = run_program<F>(P, S, prog, st);
    DEMAG_CUDA(P, cudaEventRecord(e1, st));
    DEMAG_CUDA(P, cudaEventSynchronize(e1));
    if (r != DEMAG_OK) return r;
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= 3.f;
    return DEMAG_OK;
  };
  for (int prog = 0; prog < kPrograms && s == DEMAG_OK; ++prog) {
    if (S->small[prog]) continue;  // runs on CUDA cores
    if (prog >= kChain && !S->fused) continue;
    for (int knob = 0; knob < 4 && s == DEMAG_OK; ++knob) {
      if (find_tuned(P, tune_kind(S, knob), prog)) continue;  // chosen before (a loaded cache)
      std::vector<int> cands;
      int def = 0;
      if (knob == 0) {
        def = S->host_prog[prog].bn;
        cands.push_back(def);
        for (int c = 128; c >= 64; c /= 2)
          if (c < def) cands.push_back(c);
      } else if (knob == 1) {
        def = 0;  // as many as fit
        cands = {0, 4, 3, 2};
      } else if (knob == 2) {
        def = 0;
        cands = {0, 1};
      } else {
        def = 0;
        cands = {0};
        if (S->wide[prog_axis(prog)]) cands.push_back(1);
      }
      if (cands.size() == 1) continue;
      float best = 1e30f, at_def = 0.f;
      int best_v = def;
      for (int c : cands) {
        s = set_knob(P, S, prog, knob, c);
        float ms = 0.f;
        if (s == DEMAG_OK) s = time_prog(prog, &ms);
        if (s != DEMAG_OK) break;
        if (c == def) at_def = ms;
        if (ms < best) {
          best = ms;
          best_v = c;
        }
      }
      if (s == DEMAG_OK) s = set_knob(P, S, prog, knob, best_v);
      if (s == DEMAG_OK) {
        demag_plan::Tuned t;
        t.kind = tune_kind(S, knob);
        t.key[0] = prog;
        t.key[1] = def;
        t.key[2] = 0;
        t.value = best_v;
        t.ms = best;
        t.ms_default = at_def;
        P->tuned.push_back(t);
      }
    }
  }
  // forward schedule, with every stage program tuned: fused kernel and
  // mode-3 stage against the three-stage chain
  bool have_sched = false;
  for (const demag_plan::Tuned& t : P->tuned) have_sched = have_sched || t.kind == kTuneSchedule;
  if (s == DEMAG_OK && S->fused && !have_sched) {
    float mf = 0.f, mc = 0.f;
    s = time_sched(1, &mf);
    if (s == DEMAG_OK) s = time_sched(0, &mc);
    if (s == DEMAG_OK) {
      S->sched = mc < mf ? 0 : 1;
      demag_plan::Tuned t;
      t.kind = kTuneSchedule;
      t.key[0] = 0;
      t.key[1] = 1;
      t.key[2] = 0;
      t.value = S->sched;
      t.ms = S->sched ? mf : mc;
      t.ms_default = S->sched0 ? mf : mc;
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
  const int n3 = P->n[2], M = P->M;
  TcState* S = new TcState();
  memset(S, 0, sizeof(*S));
  S->elem = prec == DEMAG_TF32X3 ? 4 : 2;
  {
    const TcGeo G = tc_geometry(P, S->elem);
    S->geo = G.g;
    for (int p = 0; p < 3; ++p) {
      S->halves[p] = G.halves[p];
      S->ld[p] = G.ld[p];
      S->ldB[p] = G.ldB[p];
      const int h = G.g.h[p];
      S->bn[p] = h >= kBN ? kBN : round_up(h, 16);
    }
  }
  const AxisGeo& geo = S->geo;
  const long long x1 = geo.ext[0], x2 = geo.ext[1], x3 = geo.ext[2];
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return false;
    S->bytes += bytes;
    return cudaMemsetAsync(*ptr, 0, bytes, st) == cudaSuccess;
  };
  const size_t e = S->elem;
  bool ok = true;
  for (int p = 0; p < 3 && ok; ++p)
    for (int h = 0; h < 2 && ok; ++h)
      ok = alloc(&S->B[p][h], (size_t)M * 2 * S->halves[p] * geo.h[p] * S->ldB[p] * e);
  for (int h = 0; h < 2 && ok; ++h) {
    ok = ok && alloc(&S->X[h], 3 * (size_t)x3 * x2 * S->ld[0] * e);
    ok = ok && alloc(&S->buf1[h], 3 * (size_t)M * x1 * x3 * S->ld[1] * e);
    ok = ok && alloc(&S->buf2[h], 3 * (size_t)M * x2 * x1 * S->ld[2] * e);
  }
  ok = ok && alloc((void**)&S->status, sizeof(int));
  ok = ok && alloc((void**)&S->counter, sizeof(int));
  {
    const int kb3 = (geo.h[2] + kRowBytes / S->elem - 1) / (kRowBytes / S->elem);
    // TF32x3 issues twice the MMAs per K of BF16x3 in stages 1-2 as well, so its
    // node sum gets half the accumulation budget
    S->pp3 = pairs_per_split(kb3, S->elem == 4 ? 200 : 400);
    // a node-sum stage on CUDA cores (single applications) accumulates in
    // round-to-nearest FP32; its groups only split the work over more blocks,
    // which a grid of few rows needs (a batched application runs the same
    // stage on tensor cores, where more groups mean more tiles and partials)
    if (n3 <= kSmallAxis && x1 * x2 < 65536) S->pp3 = std::min(S->pp3, 4);
    const int gf = (2 * M + S->pp3 - 1) / S->pp3;   // forward: 2M pairs in one sum
    const int ga = (M + S->pp3 - 1) / S->pp3;       // adjoint: M pairs per component
    const int fields = gf > 3 * ga ? gf : 3 * ga;
    S->part_fields = fields;
    ok = ok && alloc((void**)&S->part, sizeof(float) * (size_t)fields * x1 * x2 * x3);
  }
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ENOMEM, "tensor-core workspace allocation failed");
  }
  CUtensorMap mapB[3][2], mapX[2], map1[2], map2[2], out1[2], out2[2], out3, wout1[2], wout2[2], wout3;
  memset(wout1, 0, sizeof(wout1));
  memset(wout2, 0, sizeof(wout2));
  memset(&wout3, 0, sizeof(wout3));
  memset(mapB, 0, sizeof(mapB));
  memset(mapX, 0, sizeof(mapX));
  memset(map1, 0, sizeof(map1));
  memset(map2, 0, sizeof(map2));
  memset(out1, 0, sizeof(out1));
  memset(out2, 0, sizeof(out2));
  memset(&out3, 0, sizeof(out3));
  // maps of every axis, also those of at most kSmallAxis cells: a single
  // application runs those stages on CUDA cores, a batched one on tensor cores
  for (int h = 0; h < 2; ++h) {
    for (int p = 0; p < 3; ++p)
      ok = ok && make_bmap(&mapB[p][h], S->B[p][h], S->elem, geo.h[p], S->halves[p], 2 * M, S->ldB[p], S->bn[p]);
    ok = ok && make_map(&mapX[h], S->X[h], S->elem, x1, (uint64_t)(x3 * x2), 3, S->ld[0], kBM);
    ok = ok && make_map(&map1[h], S->buf1[h], S->elem, x2, (uint64_t)(x1 * x3), 3 * M, S->ld[1], kBM);
    ok = ok && make_map(&map2[h], S->buf2[h], S->elem, x3, (uint64_t)(x2 * x1), 3 * M, S->ld[2], kBM);
  }
  // epilogue stores through TMA where a warp's 32 output rows share one outer
  // index (n_inner % 32 == 0) and a 32 x 32 chunk fits the staging buffer
  // (BF16 planes, FP32 partials)
  S->tma[0] = (x2 % 32 == 0) && S->elem == 2;
  S->tma[1] = (x3 % 32 == 0) && S->elem == 2;
  S->tma[2] = (x1 % 32 == 0);
  // a whole 128-row block in one outer index: the four epilogue warps store it together
  const long long inner_of[3] = {x2, x3, x1};
  for (int st3 = 0; st3 < 3; ++st3) S->wide[st3] = S->tma[st3] && kEpiWarps == 4 && inner_of[st3] % kBM == 0;
  for (int w = 0; w < 2; ++w) {  // per-warp boxes, then the wide ones where a stage has them
    CUtensorMap* o1 = w ? wout1 : out1;
    CUtensorMap* o2 = w ? wout2 : out2;
    const uint32_t bi = w ? kBM : 32;
    for (int h = 0; h < 2; ++h) {
      if (S->tma[0] && (!w || S->wide[0]))
        ok = ok && make_out_map(&o1[h], S->buf1[h], S->elem, x2, x3, geo.h[0], S->halves[0], geo.hq[0], 3 * M,
                                S->ld[1], (uint64_t)x3 * S->ld[1], (uint64_t)(x1 * x3) * S->ld[1], bi);
      if (S->tma[1] && (!w || S->wide[1]))
        ok = ok && make_out_map(&o2[h], S->buf2[h], S->elem, x3, x1, geo.h[1], S->halves[1], geo.hq[1], 3 * M,
                                S->ld[2], (uint64_t)x1 * S->ld[2], (uint64_t)(x2 * x1) * S->ld[2], bi);
    }
    if (S->tma[2] && (!w || S->wide[2]))
      ok = ok && make_out_map(w ? &wout3 : &out3, S->part, 4, x1, x2, geo.h[2], S->halves[2], geo.hq[2],
                              S->part_fields, x1, (uint64_t)(x2 * x1), (uint64_t)(x1 * x2 * x3), bi);
  }
  if (!ok) {
    free_state(S);
    return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
  }
  // the fused forward application (mode-1 and mode-2 products in one kernel)
  CUtensorMap zA[2], zA3[2];
  memset(zA, 0, sizeof(zA));
  memset(zA3, 0, sizeof(zA3));
  {
    const int h1 = geo.h[0], h2 = geo.h[1], hq1 = geo.hq[0], hq2 = geo.hq[1];
    const int n2 = round_up(h2, 16);
    S->fused = S->elem == 2 && !P->nonuniform && geo.hq[0] && geo.hq[1] && geo.hq[2] && h1 <= 128 && h2 <= 128;
    // untuned choice (BF16x3, R = 41, CUDA events per application): the chain
    // is faster on small grids (32^3 0.072 against 0.095 ms, 80^3 0.249 against
    // 0.274, 96^3 0.325 against 0.329), the fused schedule from 112^3 on
    // (0.42 against 0.45 ms, 160^3 0.87 against 0.99, 256^3 2.14 against 3.00)
    S->sched0 = x1 * x2 * x3 >= (1LL << 20) ? 1 : 0;
    S->sched = S->sched0;
    if (S->fused) {
      S12Launch& Z = S->s12;
      for (int h = 0; h < 2 && ok; ++h) {
        void* zb = S->buf1[h];  // Z [2M][ext3][ext2][ext1] in the stage-1 workspace
        ok = ok && make_bmap(h ? &Z.t1_lo : &Z.t1_hi, S->B[0][h], 2, h1, 2, 2 * M, S->ldB[0], kBM);
        ok = ok && make_map(h ? &Z.x_lo : &Z.x_hi, S->X[h], 2, x1, (uint64_t)(x3 * x2), 3, S->ld[0], n2);
        ok = ok && make_bmap(h ? &Z.t2_lo : &Z.t2_hi, S->B[1][h], 2, h2, 2, 2 * M, S->ldB[1], n2);
        // stores clipped to the valid h1 x h2 entries of each pair of halves
        ok = ok && make_out_map(h ? &Z.z_lo : &Z.z_hi, zb, 2, h1, 2, h2, 2, hq2, (uint64_t)x3 * 2 * M, hq1, x1,
                                x2 * x1);
        ok = ok && make_map3(&zA[h], zb, x2 * x1, x3, 2 * M, x2 * x1, x3 * x2 * x1, 64, 32,
                             CU_TENSOR_MAP_SWIZZLE_128B);
        // the adjoint: 3M Z fields (buf1 holds 3M ext1 ext3 ld2 >= 3M ext3 ext2 ext1 elements)
        ok = ok && make_out_map(h ? &S->s12a.z_lo : &S->s12a.z_hi, zb, 2, h1, 2, h2, 2, hq2, (uint64_t)x3 * 3 * M,
                                hq1, x1, x2 * x1);
        ok = ok && make_map3(&zA3[h], zb, x2 * x1, x3, 3 * M, x2 * x1, x3 * x2 * x1, 64, 32,
                             CU_TENSOR_MAP_SWIZZLE_128B);
      }
      Z.M = M;
      Z.x2 = (int)x2;
      Z.x3 = (int)x3;
      Z.h1 = h1;
      Z.h2 = h2;
      Z.hq1 = hq1;
      Z.hq2 = hq2;
      Z.n2 = n2;
      Z.kb1 = (h1 + 31) / 32;
      Z.kb2 = (h2 + 31) / 32;
      Z.units = (int)x3 * M * 2;
      {  // the adjoint's launch: the same operand maps, its own Z store maps
        const CUtensorMap zh = S->s12a.z_hi, zl = S->s12a.z_lo;
        S->s12a = Z;
        S->s12a.z_hi = zh;
        S->s12a.z_lo = zl;
      }
      if (!ok) {
        free_state(S);
        return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
      }
    }
  }
  const int bk = kRowBytes / S->elem;
  demag_status s =
      build_programs(P, S, mapX, map1, map2, mapB, out1, out2, out3, wout1, wout2, wout3, zA, zA3, bk, st);
  if (s == DEMAG_OK)
    s = prec == DEMAG_TF32X3 ? prepare_form<Tf32Form>(P, S, st) : prepare_form<Bf16Form>(P, S, st);
  if (s == DEMAG_OK) s = apply_tuned(P, S);
  if (s == DEMAG_OK && P->autotune) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (cap == cudaStreamCaptureStatusNone) {
      Hd->s[form_index(prec)] = S;  // tc_sync_status reads the state through the holder
      s = prec == DEMAG_TF32X3 ? tune_programs<Tf32Form>(P, S, st) : tune_programs<Bf16Form>(P, S, st);
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
static demag_status launch_segs(demag_plan* P, const TcGroup* groups, const TcSeg* segs, int nsegs, int total_tiles,
                               int maxbn, int* counter, int* counters, int ncounters, int* status, cudaStream_t st,
                               int want_stages = 0) {
  if (total_tiles <= 0) return DEMAG_OK;
  TcLaunch L;
  L.groups = groups;
  L.segs = segs;
  L.nsegs = nsegs;
  L.total_tiles = total_tiles;
  // as many operand stages of the launch's widest N tile as fit
  L.btile = maxbn * kRowBytes;
  L.stage_bytes = (2 * kTileA + 2 * L.btile + 1023) / 1024 * 1024;
  L.nstages = std::min(kMaxStages, (kSmemMax - kSmemFixed) / L.stage_bytes);
  if (want_stages > 0) L.nstages = std::min(L.nstages, want_stages);
  const int smem_bytes = kSmemFixed + L.nstages * L.stage_bytes;
  L.tile_counter = counter;
  L.counters = counters;
  L.status = status;
  L.wait_ns = P->wait_ns;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = total_tiles < sms ? total_tiles : sms;
  // the dependency counters follow the tile counter in the same buffer when present
  DEMAG_CUDA(P, cudaMemsetAsync(counter, 0, sizeof(int) * (1 + (counters ? ncounters : 0)), st));
  DEMAG_LAUNCH(P, kFamGemmTc, st, tc_gemm_kernel<F><<<grid, kTcThreads, smem_bytes, st>>>(L));
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
  return launch_segs<F>(P, S->prog + prog, S->seg + prog, 1, S->host_prog[prog].ntiles, S->host_prog[prog].bn,
                        S->counter, nullptr, 0, S->status, st, S->nst[prog]);
}

static bool any_folded(const TcState* S) { return S->geo.hq[0] || S->geo.hq[1] || S->geo.hq[2]; }

// Operand split of one or several plans' inputs: folded plans in one
// fold_split launch, plans with no folded axis in one split_rows launch.
struct SplitLists {
  FoldList f;
  SplitList p;
  SplitLists() {
    f.count = 0;
    f.total = 0;
    p.count = 0;
    p.total = 0;
  }
};

static void add_split(SplitLists& L, demag_plan* P, TcState* S, const float* x, int fields) {
  if (any_folded(S)) {
    FoldItem& it = L.f.it[L.f.count++];
    it.x = x;
    it.hi = S->X[0];
    it.lo = S->X[1];
    it.begin = L.f.total;
    it.g = S->geo;
    it.ld1 = S->ld[0];
    long long rows = fields;
    for (int p = 1; p < 3; ++p) rows *= S->geo.hq[p] ? S->geo.hq[p] : S->geo.n[p];
    L.f.total += rows;
  } else {
    SplitItem& it = L.p.it[L.p.count++];
    it.x = x;
    it.hi = S->X[0];
    it.lo = S->X[1];
    it.begin = L.p.total;
    it.n = P->n[0];
    it.ld = S->ld[0];
    it.vec = (P->n[0] % 4 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0);
    L.p.total += (long long)fields * P->n[2] * P->n[1] * ((P->n[0] + 3) / 4);
  }
}

template <class F>
static demag_status launch_split(demag_plan* P, const SplitLists& L, cudaStream_t st) {
  if (L.f.count) {
    // rows whose first axis takes the paired path (two orbits per thread) need
    // half the threads: 64-thread blocks, twice as many resident
    bool pairs = F::kElem == 2;
    for (int i = 0; i < L.f.count; ++i) {
      const FoldItem& it = L.f.it[i];
      pairs = pairs && it.g.hq[0] && (it.g.n[0] & 3) == 0 && (reinterpret_cast<uintptr_t>(it.x) & 7) == 0;
    }
    const int threads = pairs ? 64 : 128;
    DEMAG_LAUNCH(P, kFamSplit, st,
                 fold_split_kernel<F><<<row_blocks(L.f.total, pairs ? 32 : 16), threads, 0, st>>>(L.f));
    DEMAG_LAUNCHED(P, "fold_split_kernel");
  }
  if (L.p.count) {
    DEMAG_LAUNCH(P, kFamSplit, st, split_rows_kernel<F><<<grid_blocks(L.p.total), 256, 0, st>>>(L.p));
    DEMAG_LAUNCHED(P, "split_rows_kernel");
  }
  return DEMAG_OK;
}

template <class F>
static demag_status split_input(demag_plan* P, TcState* S, const float* x, int fields, cudaStream_t st) {
  SplitLists L;
  add_split(L, P, S, x, fields);
  return launch_split<F>(P, L, st);
}

// Node-sum reduction (and unfolding) of one or several plans' partial fields.
struct ReduceLists {
  UnfoldList f;
  ReduceList p;
  ReduceLists() {
    f.count = 0;
    f.total = 0;
    p.count = 0;
    p.total = 0;
  }
};

static demag_status launch_reduce(demag_plan* P, const ReduceLists& L, cudaStream_t st) {
  if (L.f.count) {
    bool pairs = true;  // as in the fold: the paired path needs half the threads
    for (int i = 0; i < L.f.count; ++i) {
      const UnfoldItem& it = L.f.it[i];
      pairs = pairs && it.g.hq[0] && (it.g.n[0] & 3) == 0 && (reinterpret_cast<uintptr_t>(it.out) & 7) == 0;
    }
    const int threads = pairs ? 64 : 128;
    DEMAG_LAUNCH(P, kFamMisc, st,
                 unfold_reduce_kernel<<<row_blocks(L.f.total, pairs ? 24 : 16), threads, 0, st>>>(L.f));
    DEMAG_LAUNCHED(P, "unfold_reduce_kernel");
  }
  if (L.p.count) {
    DEMAG_LAUNCH(P, kFamMisc, st, reduce_parts_kernel<<<grid_blocks(L.p.total), 256, 0, st>>>(L.p));
    DEMAG_LAUNCHED(P, "reduce_parts_kernel");
  }
  return DEMAG_OK;
}

static void add_reduce(ReduceLists& L, demag_plan* P, TcState* S, int groups, int nout, float alpha, float* out) {
  if (any_folded(S)) {
    UnfoldItem& it = L.f.it[L.f.count++];
    it.part = S->part;
    it.out = out;
    it.begin = L.f.total;
    it.g = S->geo;
    it.groups = groups;
    float a = alpha;
    for (int p = 0; p < 3; ++p)
      if (S->geo.hq[p]) a *= 0.5f;
    it.alpha = a;
    L.f.total += (long long)nout * S->geo.h[1] * S->geo.h[2];
  } else {
    const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
    ReduceItem& it = L.p.it[L.p.count++];
    it.part = S->part;
    it.out = out;
    it.begin = L.p.total;
    it.N = N;
    it.groups = groups;
    it.alpha = alpha;
    it.vec = (N % 4 == 0) && (reinterpret_cast<uintptr_t>(out) % 16 == 0);
    L.p.total += it.vec ? nout * (N >> 2) : nout * N;
  }
}

static demag_status reduce_parts(demag_plan* P, TcState* S, int groups, int nout, float alpha, float* out,
                                 cudaStream_t st) {
  ReduceLists L;
  add_reduce(L, P, S, groups, nout, alpha, out);
  return launch_reduce(P, L, st);
}

// The mode-1 and mode-2 products of every slab in one launch (Z into buf1).
static demag_status run_s12(demag_plan* P, TcState* S, const S12Launch& base, cudaStream_t st, bool adj) {
  S12Launch L = base;
  L.unit_counter = S->counter;
  L.status = S->status;
  L.wait_ns = P->wait_ns;
  L.items = nullptr;
  L.unit0 = nullptr;
  L.count = 1;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = L.units < 2 * sms ? L.units : 2 * sms;  // two CTAs per SM
  DEMAG_CUDA(P, cudaMemsetAsync(S->counter, 0, sizeof(int), st));
  if (adj)
    DEMAG_LAUNCH(P, kFamGemmTc, st, tc_s12_kernel<true, false><<<grid, kS12Threads, kS12Smem, st>>>(L));
  else
    DEMAG_LAUNCH(P, kFamGemmTc, st, tc_s12_kernel<false, false><<<grid, kS12Threads, kS12Smem, st>>>(L));
  DEMAG_LAUNCHED(P, "tc_s12_kernel");
  return DEMAG_OK;
}

template <class F>
static demag_status forward_chain(demag_plan* P, TcState* S, const float* m, float* phi, cudaStream_t st) {
  demag_status s = split_input<F>(P, S, m, 3, st);
  if (S->fused && (P->fused > 0 || (P->fused < 0 && S->sched))) {
    if (s == DEMAG_OK) s = run_s12(P, S, S->s12, st);
    if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd3Z, st);
  } else {
    for (int prog = kFwd1; prog <= kFwd3 && s == DEMAG_OK; ++prog) s = run_program<F>(P, S, prog, st);
  }
  if (s != DEMAG_OK) return s;
  return reduce_parts(P, S, S->groups_fwd, 1, 1.f, phi, st);
}

template <class F>
static demag_status adjoint_chain(demag_plan* P, TcState* S, const float* y, float* g, cudaStream_t st) {
  demag_status s = split_input<F>(P, S, y, 1, st);
  if (S->fused && (P->fused > 0 || (P->fused < 0 && S->sched))) {
    // the forward's schedule: the first two transposed mode products fused
    if (s == DEMAG_OK) s = run_s12(P, S, S->s12a, st, true);
    if (s == DEMAG_OK) s = run_program<F>(P, S, kAdj3Z, st);
    if (s != DEMAG_OK) return s;
    return reduce_parts(P, S, S->groups_adj, 3, -1.f, g, st);
  }
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
  cudaFree(B->segs);
  cudaFree(B->ctr);
  cudaFree(B->s12items);
  cudaFree(B->s12unit0);
  delete B;
}

// Whether a plan's forward application takes the fused schedule.
static bool fused_schedule(const demag_plan* P, const TcState* S) {
  return S->fused && (P->fused > 0 || (P->fused < 0 && S->sched));
}

// One launch for every forward stage of `plans` (distinct, with their
// tensor-core state for `prec`): the tiles of stage 1 of all grids that run
// the chain, largest grids first, then the mode-3 stages of the grids that run
// the fused schedule (their mode-1 / mode-2 products ran before, in one
// tc_s12_kernel launch over all of them, largest first), then stage 2 and
// stage 3 of the chain grids.  Stage s of a chain grid waits for the
// completion counter of its stage s - 1 (every epilogue warp of every tile of
// that stage counts once); in this order the wait is met long before, except
// for the last grids of a stage.  (Interleaving the stages of different grids
// as a pipeline, so that a small grid's intermediates are read while still in
// L2, measured 4% slower on the 64-grid batch.)  Stages along axes of at most
// kSmallAxis cells run as tensor-core tiles here (K padded to one k-block,
// 16-wide N tiles).
demag_status tc_batch_create(demag_plan* const* plans, int count, demag_precision prec, TcBatch** out) {
  *out = nullptr;
  demag_plan* P0 = plans[0];
  TcBatch* B = new TcBatch();
  B->plans.assign(plans, plans + count);
  for (int i = 0; i < count; ++i) B->serials.push_back(plans[i]->serial);
  B->prec = (int)prec;
  // largest grids first: the dynamic tile counter then hands out their long
  // tile streams early and the small grids' tiles fill the tail of each stage
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto cells = [&](int i) { return (long long)plans[i]->n[0] * plans[i]->n[1] * plans[i]->n[2]; };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cells(a) > cells(b); });
  std::vector<TcGroup> g(3 * (size_t)count);
  std::vector<TcSeg> segs;
  std::vector<S12Launch> items;
  std::vector<int> unit0(1, 0);
  // chain grids whose last stage only is along a thin axis (films n1, n2 > 16 >= n3): that
  // stage runs on CUDA cores as in a single call, one launch for all of them after the
  // persistent one (as padded tensor-core tiles it took twice as long); other thin stages
  // stay in the persistent launch as padded tiles
  std::vector<char> thin3(count, 0);
  memset(&B->small, 0, sizeof(B->small));
  B->small.job0[0] = 0;
  B->fused.resize(count);
  for (int i = 0; i < count; ++i) {
    const TcState* S = state(plans[i], prec);
    B->fused[i] = fused_schedule(plans[i], S) ? 1 : 0;
  }
  for (int i = 0; i < count; ++i) {
    const TcState* S = state(plans[order[i]], prec);
    for (int st3 = 0; st3 < 3; ++st3) {
      g[st3 * count + i] = S->host_prog[kFwd1 + st3];
      g[st3 * count + i].o_wide = 0;  // the groups of one launch share the staging: per-warp boxes for all
    }
    if (B->fused[order[i]]) {  // slot 0 holds its mode-3 stage on Z
      g[i] = S->host_prog[kFwd3Z];
      g[i].o_wide = 0;
      items.push_back(S->s12);
      unit0.push_back(unit0.back() + S->s12.units);
    } else if (S->small[kFwd3] && !S->small[kFwd1] && !S->small[kFwd2] && B->small.count < kMaxSmallItems) {
      SmallBatch& SB = B->small;
      const SmallStage& Q = S->small_prog[kFwd3];
      thin3[i] = 1;
      SB.it[SB.count] = Q;
      SB.job0[SB.count + 1] = SB.job0[SB.count] + Q.njobs;
      SB.rowblocks = std::max(SB.rowblocks, (Q.rows + 255) / 256);
      ++SB.count;
    }
  }
  int acc = 0;
  // passes: chain stage 1, fused mode-3 stages, chain stages 2 and 3
  for (int pass = 0; pass < 4; ++pass) {
    for (int i = 0; i < count; ++i) {
      const bool fz = B->fused[order[i]] != 0;
      if (fz != (pass == 1)) continue;
      const TcState* S = state(plans[order[i]], prec);
      const int st3 = pass == 0 ? 0 : pass - 1;
      if (st3 == 2 && thin3[i]) continue;  // in the CUDA-core launch after this one
      const int gi = fz ? i : st3 * count + i;
      if (g[gi].ntiles <= 0) continue;
      TcSeg q = whole_seg(g[gi], gi, acc);
      if (!fz && st3 > 0) {
        q.dep = 2 * i + (st3 - 1);
        q.dep_target = kEpiWarps * S->host_prog[kFwd1 + st3 - 1].ntiles;
      }
      if (!fz && st3 < 2) q.done = 2 * i + st3;
      segs.push_back(q);
      acc += g[gi].ntiles;
    }
  }
  for (const TcGroup& gg : g) B->maxbn = std::max(B->maxbn, gg.bn);
  B->nsegs = (int)segs.size();
  B->total = acc;
  B->nctr = 2 * count;
  B->s12count = (int)items.size();
  B->s12units = unit0.back();
  if (cudaMalloc(&B->groups, sizeof(TcGroup) * g.size()) != cudaSuccess ||
      cudaMalloc(&B->segs, sizeof(TcSeg) * (segs.size() ? segs.size() : 1)) != cudaSuccess ||
      cudaMalloc(&B->ctr, sizeof(int) * (1 + B->nctr)) != cudaSuccess ||
      (B->s12count > 0 && (cudaMalloc(&B->s12items, sizeof(S12Launch) * items.size()) != cudaSuccess ||
                           cudaMalloc(&B->s12unit0, sizeof(int) * unit0.size()) != cudaSuccess))) {
    tc_batch_destroy(B);
    return set_error(P0, DEMAG_ENOMEM, "grouped launch descriptors: allocation failed");
  }
  cudaError_t e = cudaMemcpy(B->groups, g.data(), sizeof(TcGroup) * g.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !segs.empty())
    e = cudaMemcpy(B->segs, segs.data(), sizeof(TcSeg) * segs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && B->s12count > 0)
    e = cudaMemcpy(B->s12items, items.data(), sizeof(S12Launch) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && B->s12count > 0)
    e = cudaMemcpy(B->s12unit0, unit0.data(), sizeof(int) * unit0.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    tc_batch_destroy(B);
    return cuda_error(P0, e, "grouped launch descriptors");
  }
  *out = B;
  return DEMAG_OK;
}

// Several grids in one call: one split launch over every plan's input, one
// fused mode-1 / mode-2 launch over the grids with the fused schedule, one
// persistent launch over all remaining stages of all grids, one node-sum
// reduction launch into every plan's phi (per kMaxItems grids for the
// element-wise launches).
template <class F>
static demag_status batched_chain(const TcBatch* B, const float* const* m, float* const* phi, cudaStream_t st) {
  const demag_precision prec = (demag_precision)B->prec;
  const int count = (int)B->plans.size();
  demag_plan* P0 = B->plans[0];
  TcState* S0 = state(P0, prec);
  for (int i0 = 0; i0 < count; i0 += kMaxItems) {
    SplitLists L;
    for (int i = i0; i < count && i < i0 + kMaxItems; ++i) add_split(L, B->plans[i], state(B->plans[i], prec), m[i], 3);
    demag_status s = launch_split<F>(P0, L, st);
    if (s != DEMAG_OK) return s;
  }
  if (B->s12count > 0) {
    S12Launch L;
    memset(&L, 0, sizeof(L));
    L.units = B->s12units;
    L.unit_counter = B->ctr;  // zeroed again by the persistent launch below
    L.status = S0->status;
    L.wait_ns = P0->wait_ns;
    L.items = B->s12items;
    L.unit0 = B->s12unit0;
    L.count = B->s12count;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = L.units < 2 * sms ? L.units : 2 * sms;  // two CTAs per SM
    DEMAG_CUDA(P0, cudaMemsetAsync(B->ctr, 0, sizeof(int), st));
    DEMAG_LAUNCH(P0, kFamGemmTc, st, tc_s12_kernel<false, true><<<grid, kS12Threads, kS12Smem, st>>>(L));
    DEMAG_LAUNCHED(P0, "tc_s12_kernel");
  }
  demag_status s = launch_segs<F>(P0, B->groups, B->segs, B->nsegs, B->total, B->maxbn, B->ctr, B->ctr + 1,
                                  B->nctr, S0->status, st);
  if (s != DEMAG_OK) return s;
  if (B->small.count > 0) {
    const dim3 grid((unsigned)B->small.rowblocks, (unsigned)B->small.job0[B->small.count]);
    DEMAG_LAUNCH(P0, kFamGemmSimt, st, small_batch_kernel<F><<<grid, 256, 0, st>>>(B->small));
    DEMAG_LAUNCHED(P0, "small_batch_kernel");
  }
  for (int i0 = 0; i0 < count; i0 += kMaxItems) {
    ReduceLists L;
    for (int i = i0; i < count && i < i0 + kMaxItems; ++i) {
      TcState* S = state(B->plans[i], prec);
      add_reduce(L, B->plans[i], S, S->groups_fwd, 1, 1.f, phi[i]);
    }
    s = launch_reduce(P0, L, st);
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
  for (int i = 0; hit && i < count; ++i)
    hit = B->plans[i] == plans[i] && B->serials[i] == plans[i]->serial &&
          B->fused[i] == (fused_schedule(plans[i], state(plans[i], prec)) ? 1 : 0);
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
    const int h = S->geo.h[p];
    const size_t bytes = (size_t)M * 2 * S->halves[p] * h * S->ldB[p] * S->elem;
    for (int hl = 0; hl < 2; ++hl) {
      DEMAG_CUDA(P, cudaMalloc(&S->Bd[p][hl], bytes));
      DEMAG_CUDA(P, cudaMemsetAsync(S->Bd[p][hl], 0, bytes, st));
    }
    // dE is odd and dF even: the parity of the two types is swapped (pxor = 1)
    const long long total = (long long)M * 2 * S->halves[p] * h * h;
    DEMAG_LAUNCH(P, kFamSetup, st,
                 tc_factor_kernel<F><<<grid_blocks(total), 256, 0, st>>>(
                     M, P->glen, p, P->n[p], h, S->halves[p], S->ldB[p], 1, P->gend, P->scale,
                     (typename F::T*)S->Bd[p][0], (typename F::T*)S->Bd[p][1], nullptr, 0, 0));
    DEMAG_LAUNCHED(P, "tc_factor_kernel");
  }
  TcSeg sg[4];
  memset(sg, 0, sizeof(sg));
  for (int st3 = 0; st3 < 3; ++st3) {
    TcGroup& G = S->dprog_host[st3];
    G = S->host_prog[kFwd1 + st3];
    if (!S->small[kFwd1 + st3]) {
      const int p = st3;  // stage s contracts axis s
      for (int h = 0; h < 2; ++h)
        if (!make_bmap(h ? &G.b_lo : &G.b_hi, S->Bd[p][h], S->elem, S->geo.h[p], S->halves[p], 2 * M, S->ldB[p],
                       G.bn))
          return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
      G.pxor = 1;
    }
    S->small_dprog[st3] = S->small_prog[kFwd1 + st3];
    S->small_dprog[st3].gen = P->gend;
    S->small_dprog[st3].fac = nullptr;
    sg[st3] = whole_seg(G, 0, 0);
  }
  if (S->fused) {
    // the fused schedule with derivative factors: the mode-3 stage on Z, and
    // the fused launches with dT1 (axis 1) or dT2 (axis 2)
    TcGroup& G = S->dprog_host[3];
    G = S->host_prog[kFwd3Z];
    for (int h = 0; h < 2; ++h)
      if (!make_bmap(h ? &G.b_lo : &G.b_hi, S->Bd[2][h], S->elem, S->geo.h[2], S->halves[2], 2 * M, S->ldB[2],
                     G.bn))
        return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
    G.pxor = 1;
    sg[3] = whole_seg(G, 0, 0);
    const int h1 = S->geo.h[0], h2 = S->geo.h[1];
    S->s12d[0] = S->s12;
    S->s12d[1] = S->s12;
    bool ok = true;
    for (int h = 0; h < 2; ++h) {
      ok = ok && make_bmap(h ? &S->s12d[0].t1_lo : &S->s12d[0].t1_hi, S->Bd[0][h], 2, h1, 2, 2 * M, S->ldB[0], kBM);
      ok = ok && make_bmap(h ? &S->s12d[1].t2_lo : &S->s12d[1].t2_hi, S->Bd[1][h], 2, h2, 2, 2 * M, S->ldB[1],
                           S->s12.n2);
    }
    if (!ok) return set_error(P, DEMAG_ECUDA, "tensor map encoding failed");
    S->s12d[0].pxor1 = 1;
    S->s12d[1].pxor2 = 1;
  }
  DEMAG_CUDA(P, cudaMalloc(&S->dprog, sizeof(TcGroup) * 4));
  DEMAG_CUDA(P, cudaMalloc(&S->dseg, sizeof(sg)));
  DEMAG_CUDA(P, cudaMemcpy(S->dprog, S->dprog_host, sizeof(TcGroup) * 4, cudaMemcpyHostToDevice));
  DEMAG_CUDA(P, cudaMemcpy(S->dseg, sg, sizeof(sg), cudaMemcpyHostToDevice));
  S->field_ready = true;
  return DEMAG_OK;
}

template <class F>
static demag_status run_deriv(demag_plan* P, TcState* S, int st3, cudaStream_t st) {
  if (st3 < 3 && S->small[kFwd1 + st3]) return launch_small<F>(P, S->small_dprog[st3], st);
  return launch_segs<F>(P, S->dprog + st3, S->dseg + st3, 1, S->dprog_host[st3].ntiles, S->dprog_host[st3].bn,
                        S->counter, nullptr, 0, S->status, st);
}

// h_d[p] = -dphi/dxi_p.  The three chains share work: the stage-1 output feeds
// the directions 3 and 2, the stage-2 output direction 3, so eight stage
// launches give the three fields (three independent chains would take nine).
template <class F>
static demag_status field_chain(demag_plan* P, TcState* S, const float* m, float* hd, cudaStream_t st) {
  const long long N = (long long)P->n[0] * P->n[1] * P->n[2];
  demag_status s = prepare_field<F>(P, S, st);
  if (s == DEMAG_OK) s = split_input<F>(P, S, m, 3, st);
  if (S->fused && (P->fused > 0 || (P->fused < 0 && S->sched))) {
    // the fused schedule, once per direction (the stage-1 fields are never
    // stored, so the directions share nothing but the split input): direction
    // 3 the fused launch and the derivative mode-3 stage, directions 2 and 1
    // the fused launch with dT2 or dT1 and the mode-3 stage
    if (s == DEMAG_OK) s = run_s12(P, S, S->s12, st);
    if (s == DEMAG_OK) s = run_deriv<F>(P, S, 3, st);
    if (s == DEMAG_OK) s = reduce_parts(P, S, S->groups_fwd, 1, -1.f, hd + 2 * N, st);
    for (int dir = 1; dir >= 0 && s == DEMAG_OK; --dir) {
      s = run_s12(P, S, S->s12d[dir], st);
      if (s == DEMAG_OK) s = run_program<F>(P, S, kFwd3Z, st);
      if (s == DEMAG_OK) s = reduce_parts(P, S, S->groups_fwd, 1, -1.f, hd + dir * N, st);
    }
    return s;
  }
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

int tc_forward_schedule(const demag_plan* P, demag_precision prec) {
  const TcState* S = state(const_cast<demag_plan*>(P), prec);
  return S ? (fused_schedule(P, S) ? 1 : 0) : -1;
}

}  // namespace demag
