// Triple-product reduction on the tcgen05 tensor cores (BSP_MIXED_BF16X3 plans).
//
// The numerator of Eq. (2.7) for every kept bin is read off one dense contraction
//     M[(a,b), c] = sum_x P_ab(x) d_c(x),    P_ab = d_a d_b,
// a GEMM with M = pair rows, N = shells, K = voxels. Both operands are split into bf16 high and
// low parts, P = Ph + Pl and d = dh + dl. A pair takes two rows of an M = 128 tile, Ph and Pl,
// and the B operand is the N = 2 NP matrix [dh | dl] of the chunk's fields, so one MMA per
// 16-voxel K step gives Ph dh, Ph dl, Pl dh (and the negligible Pl dl) in four column blocks of
// an FP32 accumulator whose sum is the result (relative error about 2^-16 per product). A tile
// thus holds 64 pairs, and the instruction count per pair is that of one N = 2 NP MMA per 64
// pairs and K step.
//
// Pairs are grouped: one group (a slot) holds up to KT pairs formed from three fields f0, f1, f2,
// one pair in each of KT tiles (see TcArgs), so a generator thread loads three fields and forms
// three pair products, e.g. the triangle (a, b), (a, c), (b, c). The KT tiles of a tile group
// live side by side in one block's tensor memory and share its shared-memory field chunks.
//
// Per block (one per SM, one tile group, a contiguous voxel range), warp roles:
//   * loader warp: per 64-voxel chunk, two tiled TMA loads (high and low plane) bring NP shell
//     rows of 128 bytes with the 128-byte swizzle into an NB-stage shared-memory ring; they
//     complete on the stage's "full" mbarrier. The same bytes are the B operand of the MMAs.
//   * 16 generator warps (4 per TMEM lane quarter: 2 lane halves x 2 K-step pairs): a quad of
//     threads owns one slot, rows r (Ph) and r + 8 (Pl) of a 16-lane half, each thread four
//     voxels of every K step. It loads its slot's fields from shared memory, forms the products
//     in bf16x2 arithmetic and writes them into the tensor-memory A stage of each tile with
//     tcgen05.st .16x256b (whose lane map puts a thread's registers in rows r and r + 8). A warp
//     hands chunk i - 1's stage over while chunk i's loads are in flight, forms chunk i's
//     products and only then waits for the MMAs of chunk i - NA to free its A stage.
//   * KT MMA warps, one per tile: one thread issues the tile's 4 MMAs of a chunk into its FP32
//     accumulator and commits them to the B stage's "mma done" mbarrier (KT arrivals), which frees
//     the B stage for the loader and (NA chunks later) the A stage for the generators. One
//     issuing thread reaches an N = 64 MMA every ~45 cycles, about half the tensor core's rate;
//     several issuers keep it fed.
//   Every RUN chunks (8192 voxels) the generators read the accumulators back (tcgen05.ld) into
//   compensated FP32 sums (FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU)
//   and signal the MMA warps, whose next MMAs restart the accumulators, so FP32 sums stay short.
// Blocks keep their sums as compensated FP32 pairs; a second kernel adds them in FP64 in a fixed
// order.
// Every wait is bounded: on give-up the block raises an error flag, lets its copies and MMAs
// finish (bounded) and frees its TMEM.
#include "common.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace bsp {

namespace {

constexpr int kTcGenWarps = 16;                     // generator warps, then the loader warp, then KT MMA warps
template <int KT>
constexpr int tc_threads() { return (kTcGenWarps + 1 + KT) * 32; }
constexpr int kTcChunk = kTcVoxelChunk;             // voxels per chunk (K of one stage; one TMA box)
constexpr int kTcRun = 128;                         // chunks per FP32 accumulation run (8192 voxels)
constexpr uint32_t kTcCols = 512;                   // TMEM columns (one block per SM)
constexpr long long kWaitLimit = 1LL << 22;         // mbarrier polls before giving up
static_assert(kTcChunk == 64, "one 128-byte TMA box row per chunk");

template <int NP, int KT>
struct TcLayout {
  static constexpr int kDN = 2 * NP;                          // accumulator columns of a tile ([dh | dl])
  static constexpr int kAcc = (int)kTcCols - KT * kDN;        // first accumulator column
  static constexpr int kAStage = KT * (kTcChunk / 2);         // A columns of a stage (one bf16 per voxel)
  static constexpr int kNA = kAcc / kAStage < 4 ? kAcc / kAStage : 4;  // A stages
  static constexpr int kNB = NP == 32 ? 16 : 8;               // B stages (shared memory)
  static constexpr int kBPlane = NP * 128;                    // one plane of a chunk: NP rows x 128 bytes
  static constexpr int kBStage = 2 * kBPlane;
  static constexpr int kBarOff = kNB * kBStage;
  // barriers: full[NB], mmad[NB] (one arrival per MMA warp), gen[NA], flushed, drain; then the
  // TMEM slot and the abort flag
  static constexpr int kNumBars = 2 * kNB + kNA + 2;
  static constexpr int kBytes = 1024 + kBarOff + kNumBars * 8 + 16;  // + 1024 for the alignment
  static constexpr int kFields = KT == 1 ? 2 : 3;             // field slots a thread loads
  static_assert(kNA >= 2, "tensor memory budget");
  static_assert(kNA < kTcRun, "a run must outlast the A ring");
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static_assert(kBPlane % 1024 == 0, "boxes stay 1024-byte aligned");
};

// Poll an mbarrier; give up after Limit polls or when another warp aborted.
template <long long Limit = kWaitLimit>
__device__ __forceinline__ bool tc_wait1(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  static_assert(Limit > 0 && Limit < (1ll << 31), "poll count fits an int");
  if (ptx::mbar_try_wait(bar, parity)) return true;  // the usual case: already complete
  for (int i = 1; i < (int)Limit; ++i) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  return false;
}
// The same for a whole warp, with a warp-uniform result: every lane calls it, and a warp leaves its
// loop as one, so its warp-collective tcgen05 instructions are never run by part of a warp.
template <long long Limit = kWaitLimit>
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  return __all_sync(0xffffffffu, tc_wait1<Limit>(bar, parity, abort_flag));
}

// Self-test of the give-up path (no counterpart in the paper): one warp waits, with the loop
// above capped at kSelftestPolls polls, on an mbarrier that nothing arrives at, and raises the
// error flag as a contraction block does when a wait runs out. Nothing else is in flight: no
// copies, no tensor memory.
constexpr long long kSelftestPolls = 4096;
__global__ void tc_wait_selftest_kernel(int* error) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    ptx::mbar_init(&bar, 1);
    ptx::fence_mbar_init();
    abort_flag = 0;
  }
  __syncthreads();
  const bool done = tc_wait<kSelftestPolls>(&bar, 0u, &abort_flag);
  if (!done && threadIdx.x == 0) atomicExch(error, 1);
}

// FP32 sum kept as an unevaluated pair s + c (the rounding error of every addition goes into c),
// which holds a block's run sums to about 2^-44 without FP64 arithmetic in the loop.
struct Sum2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
  }
};

template <int NP, int KT>
__global__ void __launch_bounds__(tc_threads<KT>(), 1)
    contract_tc_kernel(TcArgs a, const __grid_constant__ CUtensorMap tmap) {
  using L = TcLayout<NP, KT>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the 128-byte swizzle repeats every 1024 bytes: boxes start on 1024-byte boundaries
  unsigned char* bs = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(bs + L::kBarOff);
  uint64_t* full = bars;
  uint64_t* mmad = bars + L::kNB;
  uint64_t* gen = bars + 2 * L::kNB;
  uint64_t* flushed = gen + L::kNA;
  uint64_t* drain = flushed + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int tg = blockIdx.x;
  const long long v_begin = (long long)blockIdx.y * a.vox_per_block;
  const long long v_end = min(v_begin + a.vox_per_block, a.nvox);
  const int nchunks = v_end > v_begin ? (int)((v_end - v_begin) / kTcChunk) : 0;

  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTcCols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < L::kNB; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&mmad[i], KT);
    }
    for (int i = 0; i < L::kNA; ++i) ptx::mbar_init(&gen[i], kTcGenWarps);
    ptx::mbar_init(flushed, kTcGenWarps);
    ptx::mbar_init(drain, KT);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tmap);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;

  if (warp == kTcGenWarps) {
    // ------------------------------------------------------------ loader
    int issued = 0;
    for (int i = 0; i < nchunks; ++i) {
      const int s = i % L::kNB;
      // stage s was last used by chunk i - NB: wait for its MMAs (they follow its generators)
      if (i >= L::kNB && !tc_wait(&mmad[s], (uint32_t)(((i - L::kNB) / L::kNB) & 1), abort_flag)) {
        failed = true;
        break;
      }
      if (lane == 0) {
        ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)L::kBStage);
        // voxel coordinate: a multiple of 64 (128 bytes), as the TMA's inner coordinate must be
        const int x = (int)(v_begin + (long long)i * kTcChunk);
        unsigned char* dst = bs + (size_t)s * L::kBStage;
        ptx::tma_load_3d(dst, &tmap, x, 0, 0, &full[s]);
        ptx::tma_load_3d(dst + L::kBPlane, &tmap, x, 0, 1, &full[s]);
      }
      ++issued;
      __syncwarp();
    }
    // no copy may still be writing shared memory when the block exits (the others may have given
    // up on them): wait, bounded, for the last NB loads
    for (int k = std::max(0, issued - L::kNB); k < issued; ++k)
      ptx::mbar_wait(&full[k % L::kNB], (uint32_t)((k / L::kNB) & 1), kWaitLimit);
  } else if (warp > kTcGenWarps) {
    // ------------------------------------------------------------ MMA issuers: warp kTcGenWarps + 1 + j
    // issues tile j (several issuing threads keep the tensor core fed at N = 2 NP)
    const int j = warp - kTcGenWarps - 1;
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, L::kDN);
    const uint64_t bdesc0 = ptx::smem_desc_sw128(ptx::smem_u32(bs), 1024u);
    const uint32_t dcol = tmem + (uint32_t)(L::kAcc + L::kDN * j);
    int sa = 0;          // i % kNA, kept as a counter (kNA need not be a power of two)
    uint32_t pa = 0;     // (i / kNA) & 1
    for (int i = 0; i < nchunks; ++i) {
      const int sb = i % L::kNB;
      const bool first = (i % kTcRun) == 0;
      if (!tc_wait(&gen[sa], pa, abort_flag) ||
          !tc_wait(&full[sb], (uint32_t)((i / L::kNB) & 1), abort_flag) ||
          (first && i > 0 && !tc_wait(flushed, (uint32_t)((i / kTcRun - 1) & 1), abort_flag))) {
        failed = true;
        break;
      }
      ptx::tc_fence_after();
      if (lane == 0) {
        // descriptor start addresses are in 16-byte units: a K step of 32 bytes adds 2
        const uint64_t bd = bdesc0 + (uint64_t)((sb * L::kBStage) >> 4);
        const uint32_t acol = tmem + (uint32_t)(L::kAStage * sa + 32 * j);
#pragma unroll
        for (int ks = 0; ks < kTcChunk / 16; ++ks)
          ptx::mma_bf16_ts(dcol, acol + (uint32_t)(8 * ks), bd + (uint64_t)(2 * ks), idesc, (first && ks == 0) ? 0u : 1u);
        ptx::mma_commit(&mmad[sb]);
      }
      __syncwarp();
      if (++sa == L::kNA) { sa = 0; pa ^= 1u; }
    }
    if (lane == 0) ptx::mma_commit(drain);  // arrives once every MMA issued above is complete
    __syncwarp();
  } else {
    // ------------------------------------------------------------ generators
    const int quarter = warp & 3;      // TMEM lanes 32 quarter .. + 31
    const int half = (warp >> 2) & 1;  // lanes 32 quarter + 16 half .. + 15
    const int kg = warp >> 3;          // K steps 2 kg, 2 kg + 1 of every chunk
    const int r = lane >> 2;           // slot row: Ph in lane r, Pl in lane r + 8 of the half
    const int t4 = lane & 3;           // voxels 4 t4 .. 4 t4 + 3 of a K step
    const int slot = quarter * 16 + half * 8 + r;
    const int4 grp = a.groups[tg * kTcSlots + slot];
    const bool sel1 = (grp.w & 1) != 0;
    const bool active = (grp.w & 2) != 0;
    const bool warp_active = __any_sync(0xffffffffu, active);
    const uint32_t lane_base = (uint32_t)(32 * quarter + 16 * half) << 16;
    // byte offsets, within a B stage's high plane, of this thread's 8 bytes of field f in K step
    // 2 kg + k: row f of the 128-byte-swizzled box, 16-byte column (2 (2 kg + k) + t4 / 2) XOR (f & 7)
    int off[L::kFields][2];
    {
      const int fs[3] = {grp.x, grp.y, grp.z};
#pragma unroll
      for (int f = 0; f < L::kFields; ++f)
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int n = fs[f];
          const int col = (2 * (2 * kg + k) + (t4 >> 1)) ^ (n & 7);
          off[f][k] = (n >> 3) * 1024 + (n & 7) * 128 + (col << 4) + ((t4 & 1) << 3);
        }
    }
    // tiles whose accumulators this warp reads back: j = kg, kg + 2; their run sums are kept as
    // compensated FP32 pairs in this block's rows of the partial-sum buffer (L2-resident, one
    // owner per entry), read, added to and written back once per run
    constexpr int kMine = (KT + 1) / 2;
    constexpr int kAccN = NP / 4;  // shells per thread and tile: 8 k + 2 t4 + e
    bool have = false;
    // Read back the accumulators of my tiles (after every MMA writing them has completed). Called
    // by whole warps (tcgen05.ld is warp-collective); only active slots keep the sums.
    // .16x256b: register 4 k + {0, 1} is lane r, columns 8 k + 2 t4 + {0, 1}; 4 k + {2, 3} the
    // same columns of lane r + 8. Column c < NP is the dh block of shell c, c >= NP the dl block.
    auto flush = [&]() {
#pragma unroll
      for (int m = 0; m < kMine; ++m) {
        const int j = kg + 2 * m;
        if (j >= KT) break;
        float v[kAccN];
#pragma unroll
        for (int c0 = 0; c0 < L::kDN; c0 += 32) {
          uint32_t w[16];
          ptx::tmem_ld_16x256b_x4(tmem + lane_base + (uint32_t)(L::kAcc + L::kDN * j + c0), w);
          ptx::tmem_ld_wait();
          const int sb0 = (c0 % NP) / 8;  // first 8-shell group of this block
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float x = __uint_as_float(w[4 * k + e]) + __uint_as_float(w[4 * k + 2 + e]);
              v[2 * (sb0 + k) + e] = c0 < NP ? x : v[2 * (sb0 + k) + e] + x;
            }
        }
        if (!active) continue;
        float2* out = a.partial + ((((size_t)blockIdx.y * a.n_tg + tg) * KT + j) * kTcSlots + slot) * NP;
#pragma unroll
        for (int k = 0; k < NP / 8; ++k)
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            Sum2 t;
            if (have) { const float2 o = out[8 * k + 2 * t4 + e]; t.s = o.x; t.c = o.y; }
            t.add(v[2 * k + e]);
            out[8 * k + 2 * t4 + e] = make_float2(t.s, t.c);
          }
      }
      have = true;
    };
    // Hand a finished A stage to the MMA warp once its tensor-memory stores have landed. Done one
    // chunk late, so the store latency overlaps the next chunk's arithmetic. One arrival per warp.
    auto publish = [&](int s) {
      ptx::tmem_st_wait();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&gen[s]);
    };
    int sa = 0, sa_prev = L::kNA - 1;  // i % kNA and (i - 1) % kNA, kept as counters
    for (int i = 0; i < nchunks; ++i) {
      const int sb = i % L::kNB;
      if (!tc_wait(&full[sb], (uint32_t)((i / L::kNB) & 1), abort_flag)) {
        *abort_flag = 1;
        failed = true;
        break;
      }
      const unsigned char* st = bs + (size_t)sb * L::kBStage;
      // this slot's fields for 4 voxels of each of 2 K steps (high and low planes)
      uint2 fh[2][L::kFields], fl[2][L::kFields];
      if (warp_active) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int f = 0; f < L::kFields; ++f) {
            fh[k][f] = *reinterpret_cast<const uint2*>(st + off[f][k]);
            fl[k][f] = *reinterpret_cast<const uint2*>(st + L::kBPlane + off[f][k]);
          }
      }
      // the previous chunk's A stores have landed while the loads were in flight: hand it over
      if (i > 0) publish(sa_prev);
      // A operand: the slot's KT pair products; tile 0 (f0, s ? f1 : f0), 1 (f0, f2), 2 (f1, f2)
      uint32_t pv[KT][8];
      if (warp_active) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
          for (int j = 0; j < KT; ++j) {
            const int ia = j == 2 ? 1 : 0;
            const int ib = j == 0 ? 1 : 2;
            uint2 bh = fh[k][ib < L::kFields ? ib : 0], bl = fl[k][ib < L::kFields ? ib : 0];
            if (j == 0 && !sel1) { bh = fh[k][0]; bl = fl[k][0]; }
            ptx::bf16x2_pair_product(fh[k][ia].x, fl[k][ia].x, bh.x, bl.x, pv[j][4 * k + 0], pv[j][4 * k + 2]);
            ptx::bf16x2_pair_product(fh[k][ia].y, fl[k][ia].y, bh.y, bl.y, pv[j][4 * k + 1], pv[j][4 * k + 3]);
          }
      }
      if (i > 0 && i % kTcRun == 0) {
        // chunk i - 1 closed a run: wait for its MMAs (and with them every earlier one), read
        // the accumulators back, then let the MMA warps restart them
        const int j = i - 1;
        if (!tc_wait(&mmad[j % L::kNB], (uint32_t)((j / L::kNB) & 1), abort_flag)) {
          *abort_flag = 1;
          failed = true;
          break;
        }
        ptx::tc_fence_after();
        if (warp_active) flush();
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(flushed);
      }
      if (i >= L::kNA) {
        const int j = i - L::kNA;  // the chunk that last used A stage sa
        if (!tc_wait(&mmad[j % L::kNB], (uint32_t)((j / L::kNB) & 1), abort_flag)) {
          *abort_flag = 1;
          failed = true;
          break;
        }
      }
      ptx::tc_fence_after();
      if (warp_active) {
#pragma unroll
        for (int j = 0; j < KT; ++j)
          ptx::tmem_st_16x256b_x2(tmem + lane_base + (uint32_t)(L::kAStage * sa + 32 * j + 16 * kg), pv[j]);
      }
      sa_prev = sa;
      if (++sa == L::kNA) sa = 0;
    }
    if (!failed && nchunks > 0) publish((nchunks - 1) % L::kNA);
    if (!failed && nchunks > 0) {
      const int last = nchunks - 1;
      if (tc_wait(&mmad[last % L::kNB], (uint32_t)((last / L::kNB) & 1), abort_flag)) {
        ptx::tc_fence_after();
        if (warp_active) flush();
      } else {
        failed = true;
      }
    }
    if (failed) ptx::tmem_st_wait();
    if (nchunks == 0 && active) {
      // a block without voxels (a short x-slab of a budgeted plan) still owns its partial sums
#pragma unroll
      for (int m = 0; m < kMine; ++m) {
        const int j = kg + 2 * m;
        if (j >= KT) break;
        float2* out = a.partial + ((((size_t)blockIdx.y * a.n_tg + tg) * KT + j) * kTcSlots + slot) * NP;
#pragma unroll
        for (int k = 0; k < NP / 8; ++k)
#pragma unroll
          for (int e = 0; e < 2; ++e) out[8 * k + 2 * t4 + e] = make_float2(0.f, 0.f);
      }
    }
  }
  if (failed) {
    *abort_flag = 1;
    atomicExch(a.error, 1);
  }
  // every MMA this block issued has completed before tensor memory is released (bounded)
  if (warp > kTcGenWarps) ptx::mbar_wait(drain, 0u, kWaitLimit);
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTcCols);
  }
}

// hi[i] / lo[i]: the bf16 split of the value pair src[i] (hi at dst, lo at dst + n).
__global__ void split_fields_kernel(const float2* __restrict__ src, uint32_t* __restrict__ dst, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    uint32_t h, l;
    ptx::split_bf16x2(ptx::f2_pack(v.x, v.y), h, l);
    dst[i] = h;
    dst[n + i] = l;
  }
}

// msum[t] for the bins of all levels: lane l adds blocks y = l, l + 32, ... in order, then the
// warp adds its 32 partial sums by a fixed butterfly, so the result does not depend on timing.
__global__ void reduce_tc_all_kernel(const TcBin* __restrict__ bins, int n, double* __restrict__ msum, int accumulate) {
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const TcBin b = bins[t];
  double s = 0.0;
  for (int y = lane; y < b.gridy; y += 32) {
    const float2 v = b.partial[(long long)y * b.stride + b.off];
    s += (double)v.x + (double)v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) msum[t] = accumulate ? msum[t] + b.scale * s : b.scale * s;
}

}  // namespace

bsp_status launch_reduce_tc_all(const TcBin* bins, int n, double* msum, cudaStream_t s, bool accumulate) {
  if (n == 0) return BSP_OK;
  const long long threads = 32LL * n;
  reduce_tc_all_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(bins, n, msum, accumulate ? 1 : 0);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

int tc_padded_shells(int ns) { return ns <= 32 ? 32 : 64; }

bsp_status launch_wait_selftest(int* error, cudaStream_t s) {
  tc_wait_selftest_kernel<<<1, 32, 0, s>>>(error);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

size_t tc_partial_entries(int n_tg, int kt, int gridy, int np) {
  return (size_t)gridy * n_tg * kt * kTcSlots * np;
}

namespace {
template <int NP, int KT>
bsp_status launch_tc(const TcArgs& a, const CUtensorMap* tmap, cudaStream_t s) {
  const int smem = TcLayout<NP, KT>::kBytes;
  BSP_CUDA(cudaFuncSetAttribute(contract_tc_kernel<NP, KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  contract_tc_kernel<NP, KT><<<dim3(a.n_tg, a.gridy), tc_threads<KT>(), smem, s>>>(a, *tmap);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}
}  // namespace

bsp_status launch_contract_tc(const TcArgs& a, const CUtensorMap* tmap, cudaStream_t s) {
  if (a.n_tg == 0) return BSP_OK;
  if (a.nvox % kTcChunk != 0 || a.vox_per_block % kTcChunk != 0 || a.vox_per_block <= 0)
    return fail_c(BSP_ERR_INVALID_ARG, "tensor-core contraction: voxel ranges must be multiples of 64");
  if (a.np == 32) {
    if (a.kt == 1) return launch_tc<32, 1>(a, tmap, s);
    if (a.kt == 2) return launch_tc<32, 2>(a, tmap, s);
    if (a.kt == 3) return launch_tc<32, 3>(a, tmap, s);
  } else if (a.np == 64) {
    if (a.kt == 1) return launch_tc<64, 1>(a, tmap, s);
    if (a.kt == 2) return launch_tc<64, 2>(a, tmap, s);
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "tensor-core contraction: unsupported shell count or tile group");
}

bsp_status launch_split_fields(const float* src, uint32_t* dst, long long n_words, int n_sm, cudaStream_t s) {
  if (n_words == 0) return BSP_OK;
  const long long blocks = std::min<long long>((n_words + 255) / 256, 16LL * n_sm);
  split_fields_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<const float2*>(src), dst, n_words);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
}  // namespace

bsp_status encode_split_map(CUtensorMap* map, void* base, long long nvox, int rows, int np) {
  static EncodeTiledFn fn = nullptr;
  if (fn == nullptr) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    BSP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || f == nullptr)
      return fail_c(BSP_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    fn = reinterpret_cast<EncodeTiledFn>(f);
  }
  if (rows > np || (nvox % kTcChunk) != 0 || (reinterpret_cast<uintptr_t>(base) & 15) != 0)
    return fail_c(BSP_ERR_INVALID_ARG, "split fields: bad layout for the tensor map");
  // dims (voxel, shell, part); rows >= `rows` of a box read as zero
  const cuuint64_t dims[3] = {(cuuint64_t)nvox, (cuuint64_t)rows, 2};
  const cuuint64_t strides[2] = {(cuuint64_t)nvox * 2, (cuuint64_t)rows * (cuuint64_t)nvox * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kTcChunk, (cuuint32_t)np, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail_c(BSP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return BSP_OK;
}

}  // namespace bsp
