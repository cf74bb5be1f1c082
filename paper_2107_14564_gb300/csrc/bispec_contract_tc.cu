// Triple-product reduction on the tcgen05 tensor cores (BSP_MIXED_BF16X3 plans).
//
// The numerator of Eq. (2.7) for every kept bin is read off one dense contraction
//     M[(a,b), c] = sum_x P_ab(x) d_c(x),    P_ab = d_a d_b,
// a GEMM with M = pairs (128 per tile), N = shells (padded to NP), K = voxels. Both operands are
// split into bf16 high and low parts, P = Ph + Pl and d = dh + dl, and the MMAs accumulate
// (Ph + Pl)(dh + dl) in FP32 (relative error about 2^-16 per product). With NP = 32 the high and
// low rows of the fields form one N = 64 operand [dh | dl]: two MMAs per K step (Ph and Pl) fill
// two 32-column halves whose sum is the result; an N = 32 MMA costs about as long as an N = 64
// one, so this is a third fewer MMA instructions. With NP = 64 three MMAs per K step accumulate
// Ph dh + Ph dl + Pl dh.
//
// The fields arrive already split (two bf16 planes, written so by the Z pass). Per block (one per
// SM, one M tile of 128 pair rows, a contiguous voxel range), warp roles:
//   * loader warp: per 128-voxel chunk, four tiled TMA loads (two 64-voxel halves, high and low
//     plane each) bring the chunk's fields, NP shell rows of 128 bytes with the 128-byte swizzle,
//     into an NB-stage shared-memory ring, laid out [half][plane][row]; they complete on the
//     stage's "full" mbarrier. The same bytes are the B operand of the MMAs.
//   * 16 generator warps (4 per TMEM lane quarter, 32 voxels each): every thread owns one pair
//     row (its TMEM lane). It forms the pair products from the split fields in shared memory
//     (bf16x2 arithmetic, two voxels per instruction) and writes the A operand straight into
//     tensor memory with tcgen05.st. A lane quarter with no pair row does no work. A warp forms
//     chunk i's products first and only then waits for the MMAs of chunk i - NA to free its A
//     stage, so the products overlap those MMAs.
//   * MMA warp: one thread issues the MMAs of a chunk (8 K steps) into an FP32 accumulator in
//     tensor memory and commits them to the B stage's "mma done" mbarrier, which frees the B
//     stage for the loader and (NA chunks later) the A stage for the generators.
//   A lives in a 3-stage tensor-memory ring, B in the shared-memory ring, so loads, generation
//   and MMAs of consecutive chunks overlap; warps hand stages over through mbarriers only.
//   Every 32 chunks (4096 voxels) the generators read the accumulator back (tcgen05.ld) into FP64
//   registers while a second accumulator takes over, so FP32 sums stay short.
// Blocks write FP64 partial sums; a second kernel adds them in a fixed order.
// Every wait is bounded: on give-up the block raises an error flag, drains and frees its TMEM.
#include "common.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace bsp {

namespace {

constexpr int kTcGenWarps = 16;                     // generator warps
constexpr int kTcThreads = (kTcGenWarps + 2) * 32;  // + loader warp + MMA warp
constexpr int kTcChunk = kTcVoxelChunk;             // voxels per chunk (K of one stage)
constexpr int kTcBox = 64;                          // voxels per TMA box (128 bytes of bf16)
constexpr int kTcRun = 32;                          // chunks per FP32 accumulation run (4096 voxels)
constexpr int kTcNA = 3;                            // A operand stages (tensor memory)
constexpr uint32_t kTcCols = 512;                   // TMEM columns (one block per SM)
constexpr long long kWaitLimit = 1LL << 22;         // mbarrier polls before giving up
static_assert(kTcNA < kTcRun, "a run must outlast the operand ring");
static_assert(kTcChunk == 2 * kTcBox, "two boxes per chunk");

template <int NP>
struct TcSmem {
  static constexpr int kNB = NP == 32 ? 8 : 6;     // B stages (shared memory)
  static constexpr int kBHalf = NP * 128;          // one box: NP rows x 128 bytes (one plane)
  static constexpr int kBPart = kBHalf;            // high -> low plane of a half
  static constexpr int kBHalfStride = 2 * kBHalf;  // 64-voxel half -> next half
  static constexpr int kBStage = 2 * kBHalfStride; // two halves
  static constexpr bool kJoint = NP == 32;         // [dh | dl] as one N = 64 operand
  static constexpr int kDN = kJoint ? 2 * NP : NP; // accumulator columns of one run
  static constexpr int kBarOff = kNB * kBStage;
  // barriers: full[NB], mmad[NB], gen[NA], drain; then the TMEM slot and the abort flag
  static constexpr int kNumBars = 2 * kNB + kTcNA + 1;
  static constexpr int kBytes = 1024 + kBarOff + kNumBars * 8 + 16;  // + 1024 for the alignment
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
  static_assert(kBHalf % 1024 == 0, "boxes stay 1024-byte aligned");
};

// Poll an mbarrier; give up after kWaitLimit polls or when another warp aborted.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (long long i = 0; i < kWaitLimit; ++i) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    if ((i & 255) == 255 && *abort_flag) return false;
  }
  return false;
}

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 1)
    contract_tc_kernel(TcArgs a, const __grid_constant__ CUtensorMap tmap) {
  using L = TcSmem<NP>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the 128-byte swizzle repeats every 1024 bytes: boxes start on 1024-byte boundaries
  unsigned char* bs = smem_raw + ((1024u - (ptx::smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* bars = reinterpret_cast<uint64_t*>(bs + L::kBarOff);
  uint64_t* full = bars;
  uint64_t* mmad = bars + L::kNB;
  uint64_t* gen = bars + 2 * L::kNB;
  uint64_t* drain = gen + kTcNA;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int mtile = blockIdx.x;
  const long long v_begin = (long long)blockIdx.y * a.vox_per_block;
  const long long v_end = min(v_begin + a.vox_per_block, a.nvox);
  const int nchunks = v_end > v_begin ? (int)((v_end - v_begin) / kTcChunk) : 0;

  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTcCols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    // generator warps that take part: 4 per lane quarter holding at least one pair row
    int quarters = 0;
    for (int q = 0; q < 4; ++q) {
      bool any = false;
      for (int r = 0; r < 32; ++r) any |= a.pair_ab[mtile * 128 + 32 * q + r].x >= 0;
      quarters += any;
    }
    for (int i = 0; i < L::kNB; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&mmad[i], 1);
    }
    for (int i = 0; i < kTcNA; ++i) ptx::mbar_init(&gen[i], 4 * (quarters > 0 ? quarters : 1));
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
    ptx::prefetch_tmap(&tmap);
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: A stage s at [128 s, 128 s + 128) (hi +0..63, lo +64..127), s < 3;
  // FP32 accumulators of run parity r at [384 + DN r, 384 + DN (r + 1)).
  constexpr uint32_t kAcols = kTcChunk;  // 32-bit columns of one A stage (hi and lo halves)
  constexpr uint32_t kDcol = kAcols * kTcNA;
  static_assert(kDcol + 2 * L::kDN <= kTcCols, "tensor memory budget");
  bool failed = false;

  if (warp == kTcGenWarps) {
    // ------------------------------------------------------------ loader
    for (int i = 0; i < nchunks; ++i) {
      const int s = i % L::kNB;
      // stage s was last used by chunk i - NB: wait for its MMAs
      if (i >= L::kNB && !tc_wait(&mmad[s], (uint32_t)(((i - L::kNB) / L::kNB) & 1), abort_flag)) {
        failed = true;
        break;
      }
      if (lane == 0) {
        ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)L::kBStage);
        // voxel coordinate: a multiple of 64 (128 bytes), as the TMA's inner coordinate must be
        const int x = (int)(v_begin + (long long)i * kTcChunk);
        unsigned char* dst = bs + (size_t)s * L::kBStage;
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            ptx::tma_load_3d(dst + h * L::kBHalfStride + part * L::kBPart, &tmap, x + kTcBox * h, 0, part, &full[s]);
      }
      __syncwarp();
    }
  } else if (warp == kTcGenWarps + 1) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, L::kDN);
    for (int i = 0; i < nchunks; ++i) {
      const int sa = i % kTcNA;
      const int sb = i % L::kNB;
      if (!tc_wait(&gen[sa], (uint32_t)((i / kTcNA) & 1), abort_flag) ||
          !tc_wait(&full[sb], (uint32_t)((i / L::kNB) & 1), abort_flag)) {
        failed = true;
        break;
      }
      ptx::tc_fence_after();
      if (lane == 0) {
        const int run = i / kTcRun;
        const bool first = (i % kTcRun) == 0;
        const uint32_t dcol = tmem + kDcol + (uint32_t)(L::kDN * (run & 1));
        const uint32_t b0 = ptx::smem_u32(bs + (size_t)sb * L::kBStage);
#pragma unroll
        for (int ks = 0; ks < kTcChunk / 16; ++ks) {
          const uint32_t ahi = tmem + (uint32_t)(kAcols * sa + 8 * ks);
          const uint32_t alo = ahi + kAcols / 2;
          // K step ks: half ks / 4, 32-byte column step ks % 4 inside the swizzle atom
          const uint32_t off = (uint32_t)((ks >> 2) * L::kBHalfStride + (ks & 3) * 32);
          const uint64_t dh = ptx::smem_desc_sw128(b0 + off, 1024u);  // with kJoint: rows dh then dl
          ptx::mma_bf16_ts(dcol, ahi, dh, idesc, (first && ks == 0) ? 0u : 1u);
          if constexpr (L::kJoint) {
            ptx::mma_bf16_ts(dcol, alo, dh, idesc, 1u);
          } else {
            const uint64_t dl = ptx::smem_desc_sw128(b0 + off + L::kBPart, 1024u);
            ptx::mma_bf16_ts(dcol, ahi, dl, idesc, 1u);
            ptx::mma_bf16_ts(dcol, alo, dh, idesc, 1u);
          }
        }
        ptx::mma_commit(&mmad[sb]);
      }
      __syncwarp();
    }
    if (lane == 0) ptx::mma_commit(drain);  // arrives once every MMA issued above is complete
    __syncwarp();
  } else {
    // ------------------------------------------------------------ generators
    const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
    const int sub = warp >> 2;     // voxels [32 sub, 32 sub + 32) of a chunk
    const int row = 32 * quarter + lane;
    const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
    const int2 ab = a.pair_ab[mtile * 128 + row];
    const bool active = __any_sync(0xffffffffu, ab.x >= 0);
    // padding rows hold (-a - 1, -b - 1) of a real row of their 8-row phase (a broadcast read);
    // their accumulator rows are never read (a D row depends only on its own A row)
    const int ra = ab.x >= 0 ? ab.x : -ab.x - 1;
    const int rb = ab.x >= 0 ? ab.y : -ab.y - 1;
    constexpr int kCols = NP / 4;  // accumulator columns this thread flushes
    double acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = 0.0;
    auto flush = [&](int run) {
      const uint32_t dcol = kDcol + (uint32_t)(L::kDN * (run & 1)) + (uint32_t)(kCols * sub);
#pragma unroll
      for (int j0 = 0; j0 < kCols; j0 += 8) {
        uint32_t v[8], w[8];
        ptx::tmem_ld8(tmem + lane_base + dcol + j0, v);
        if constexpr (L::kJoint) ptx::tmem_ld8(tmem + lane_base + dcol + NP + j0, w);  // the dl half
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          acc[j0 + j] += (double)__uint_as_float(v[j]);
          if constexpr (L::kJoint) acc[j0 + j] += (double)__uint_as_float(w[j]);
        }
      }
    };
    // Hand a finished A stage to the MMA warp once its tensor-memory stores have landed. Done one
    // chunk late, so the store latency overlaps the next chunk's arithmetic. One arrival per warp.
    auto publish = [&](int s) {
      ptx::tmem_st_wait();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&gen[s]);
    };
    // Field n, voxels [32 sub + 8 m, +8) of a plane: row n of half sub / 2 (8-row atoms of 1024
    // bytes, 128-byte rows), 16-byte column (4 (sub & 1) + m) XOR (n & 7) (the TMA's swizzle).
    const int half = sub >> 1;
    const int j0 = (sub & 1) * 4;
    const int rowa = half * L::kBHalfStride + (ra >> 3) * 1024 + (ra & 7) * 128;
    const int rowb = half * L::kBHalfStride + (rb >> 3) * 1024 + (rb & 7) * 128;
    const int xa = ra & 7, xb = rb & 7;
    for (int i = 0; active && i < nchunks; ++i) {
      const int sa = i % kTcNA;
      const int sb = i % L::kNB;
      if (!tc_wait(&full[sb], (uint32_t)((i / L::kNB) & 1), abort_flag)) {
        *abort_flag = 1;
        failed = true;
        break;
      }
      const unsigned char* st = bs + (size_t)sb * L::kBStage;
      // A operand: 32 pair products of this row from the split fields a and b
      uint32_t hv[16], lv[16];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int ca = ((j0 + m) ^ xa) << 4;
        const int cb = ((j0 + m) ^ xb) << 4;
        const uint4 ah = *reinterpret_cast<const uint4*>(st + rowa + ca);
        const uint4 al = *reinterpret_cast<const uint4*>(st + L::kBPart + rowa + ca);
        const uint4 bh = *reinterpret_cast<const uint4*>(st + rowb + cb);
        const uint4 bl = *reinterpret_cast<const uint4*>(st + L::kBPart + rowb + cb);
        ptx::bf16x2_pair_product(ah.x, al.x, bh.x, bl.x, hv[4 * m + 0], lv[4 * m + 0]);
        ptx::bf16x2_pair_product(ah.y, al.y, bh.y, bl.y, hv[4 * m + 1], lv[4 * m + 1]);
        ptx::bf16x2_pair_product(ah.z, al.z, bh.z, bl.z, hv[4 * m + 2], lv[4 * m + 2]);
        ptx::bf16x2_pair_product(ah.w, al.w, bh.w, bl.w, hv[4 * m + 3], lv[4 * m + 3]);
      }
      if (i > 0) publish((i - 1) % kTcNA);
      if (i >= kTcNA) {
        const int j = i - kTcNA;  // the chunk that last used A stage sa
        if (!tc_wait(&mmad[j % L::kNB], (uint32_t)((j / L::kNB) & 1), abort_flag)) {
          *abort_flag = 1;
          failed = true;
          break;
        }
      }
      ptx::tc_fence_after();
      // The MMAs of chunk i - NA, the first chunk of run r, have completed, and with them every
      // MMA of run r - 1 (MMAs complete in issue order): read that run's accumulator now. Its
      // columns are next written by run r + 1, which starts only after chunk (r + 1) * RUN has
      // been generated, later in this loop.
      if (i >= kTcRun && i % kTcRun == kTcNA) flush(i / kTcRun - 1);
      const uint32_t acol = (uint32_t)(kAcols * sa + 16 * sub);
      ptx::tmem_st16(tmem + lane_base + acol, hv);
      ptx::tmem_st16(tmem + lane_base + acol + kAcols / 2, lv);
    }
    if (active && !failed && nchunks > 0) publish((nchunks - 1) % kTcNA);
    if (active && !failed && nchunks > 0) {
      const int last = nchunks - 1;
      if (tc_wait(&mmad[last % L::kNB], (uint32_t)((last / L::kNB) & 1), abort_flag)) {
        ptx::tc_fence_after();
        const int last_run = last / kTcRun;
        // the previous run is still unread if the last run has fewer than NA + 1 chunks
        if (last_run >= 1 && last % kTcRun < kTcNA) flush(last_run - 1);
        flush(last_run);
      } else {
        failed = true;
      }
    }
    if (failed) ptx::tmem_st_wait();
    if (active && !failed) {
      double* out = a.partial + (((size_t)blockIdx.y * a.n_mtiles + mtile) * 128 + row) * NP + kCols * sub;
#pragma unroll
      for (int j = 0; j < kCols; ++j) out[j] = acc[j];
    }
  }
  if (failed) {
    *abort_flag = 1;
    atomicExch(a.error, 1);
  }
  // every MMA this block issued has completed before tensor memory is released (bounded)
  if (warp == kTcGenWarps + 1) ptx::mbar_wait(drain, 0u, kWaitLimit);
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
__global__ void reduce_tc_all_kernel(const TcBin* __restrict__ bins, int n, double* __restrict__ msum) {
  const int t = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n) return;
  const TcBin b = bins[t];
  double s = 0.0;
  for (int y = lane; y < b.gridy; y += 32) s += b.partial[(long long)y * b.stride + b.off];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) msum[t] = b.scale * s;
}

}  // namespace

bsp_status launch_reduce_tc_all(const TcBin* bins, int n, double* msum, cudaStream_t s) {
  if (n == 0) return BSP_OK;
  const long long threads = 32LL * n;
  reduce_tc_all_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(bins, n, msum);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

int tc_padded_shells(int ns) { return ns <= 32 ? 32 : 64; }

size_t tc_partial_doubles(int n_mtiles, int gridy, int np) { return (size_t)gridy * n_mtiles * 128 * np; }

bsp_status launch_contract_tc(const TcArgs& a, const CUtensorMap* tmap, cudaStream_t s) {
  if (a.n_mtiles == 0) return BSP_OK;
  dim3 grid(a.n_mtiles, a.gridy);
  if (a.np == 32) {
    const int smem = TcSmem<32>::kBytes;
    BSP_CUDA(cudaFuncSetAttribute(contract_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    contract_tc_kernel<32><<<grid, kTcThreads, smem, s>>>(a, *tmap);
  } else if (a.np == 64) {
    const int smem = TcSmem<64>::kBytes;
    BSP_CUDA(cudaFuncSetAttribute(contract_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    contract_tc_kernel<64><<<grid, kTcThreads, smem, s>>>(a, *tmap);
  } else {
    return fail_c(BSP_ERR_NOT_SUPPORTED, "tensor-core contraction supports at most 64 shells");
  }
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
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
  const cuuint32_t box[3] = {(cuuint32_t)kTcBox, (cuuint32_t)np, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail_c(BSP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return BSP_OK;
}

}  // namespace bsp
