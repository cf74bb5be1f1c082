// Triple-product reduction on the tcgen05 tensor cores (BSP_MIXED_BF16X3 plans).
//
// The numerator of Eq. (2.7) for every kept bin is read off one dense contraction
//     M[(a,b), c] = sum_x P_ab(x) d_c(x),    P_ab = d_a d_b,
// a GEMM with M = pairs (128 per tile), N = shells (padded to NP), K = voxels. Both operands are
// split into bf16 high and low parts, P = Ph + Pl and d = dh + dl, and three MMAs per K step
// accumulate Ph dh + Ph dl + Pl dh in FP32 (relative error about 2^-16 per product).
//
// Per block (one per SM, one M tile of 128 pair rows, a contiguous voxel range), warp roles:
//   * loader warp: one 1D bulk copy (TMA) per shell row brings the FP32 fields of a 64-voxel
//     chunk into a 4-stage shared-memory ring, completing on a "full" mbarrier;
//   * 16 generator warps (4 per TMEM lane quarter, 16 voxels each): every thread owns one pair
//     row (its TMEM lane). It forms the pair products on CUDA cores (packed FP32x2), splits them
//     into bf16 high and low parts and writes the A operand straight into tensor memory with
//     tcgen05.st; the first 8 warps also split the fields into the bf16 B operand in shared
//     memory (K-major core matrices of 8 rows x 16 bytes, no swizzle);
//   * MMA warp: one thread issues 12 MMAs per chunk (4 K steps x 3 products) into an FP32
//     accumulator in tensor memory and commits them to the stage's "mma done" mbarrier.
//   A and B live in a 4-stage ring (tensor memory / shared memory), so generation of later
//   chunks overlaps the MMAs of earlier ones; warps hand stages over through mbarriers only.
//   Every 16 chunks (1024 voxels) the generators read the accumulator back (tcgen05.ld) into FP64
//   registers while a second accumulator takes over, so FP32 sums stay short.
// Blocks write FP64 partial sums; a second kernel adds them in a fixed order.
// Every wait is bounded: on give-up the block raises an error flag, drains and frees its TMEM.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace bsp {

namespace {

constexpr int kTcGenWarps = 16;                   // generator warps
constexpr int kTcThreads = (kTcGenWarps + 2) * 32;  // + loader warp + MMA warp
constexpr int kTcGen = kTcGenWarps * 32;            // generator threads
constexpr int kTcChunk = kTcVoxelChunk;             // voxels per chunk (K of one stage)
constexpr int kTcRun = 32;                          // chunks per FP32 accumulation run (4096 voxels)
constexpr int kTcFld = kTcChunk + 4;                // padded FP32 row in shared memory (floats)
constexpr int kTcNS = 3;                            // A/B operand stages
constexpr uint32_t kTcCols = 512;                   // TMEM columns (one block per SM)
constexpr long long kWaitLimit = 1LL << 22;         // mbarrier polls before giving up
static_assert(kTcNS < kTcRun, "a run must outlast the operand ring");

template <int NP>
struct TcSmem {
  static constexpr int kNF = NP == 32 ? 4 : 2;                    // FP32 field stages
  static constexpr int kFsStage = (NP + 1) * kTcFld * 4;          // FP32 stage; row NP stays zero
  static constexpr int kBPart = NP * kTcChunk * 2;                // one bf16 operand part
  static constexpr int kBsOff = (kNF * kFsStage + 1023) / 1024 * 1024;
  static constexpr int kBarOff = kBsOff + kTcNS * 2 * kBPart;
  // barriers: full[NF], empty[NF], gen[NS], mma[NS], drain; then the TMEM slot and abort flag
  static constexpr int kNumBars = 2 * kNF + 2 * kTcNS + 1;
  static constexpr int kBytes = kBarOff + kNumBars * 8 + 16;
  static_assert(kBytes <= 227 * 1024, "shared memory budget");
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
__global__ void __launch_bounds__(kTcThreads, 1) contract_tc_kernel(TcArgs a) {
  using L = TcSmem<NP>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* fs = reinterpret_cast<float*>(smem);
  unsigned char* bs = smem + L::kBsOff;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* full = bars;
  uint64_t* empty = bars + L::kNF;
  uint64_t* gen = bars + 2 * L::kNF;
  uint64_t* mma = bars + 2 * L::kNF + kTcNS;
  uint64_t* drain = bars + 2 * L::kNF + 2 * kTcNS;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kBarOff + L::kNumBars * 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + L::kBarOff + L::kNumBars * 8 + 4);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int mtile = blockIdx.x;
  const long long v_begin = (long long)blockIdx.y * a.vox_per_block;
  const long long v_end = min(v_begin + a.vox_per_block, a.nvox);
  const int nchunks = v_end > v_begin ? (int)((v_end - v_begin) / kTcChunk) : 0;

  // FP32 rows >= ns are never loaded and must read as 0
  for (int i = tid; i < L::kNF * L::kFsStage / 16; i += kTcThreads)
    reinterpret_cast<float4*>(fs)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTcCols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < L::kNF; ++i) {
      ptx::mbar_init(&full[i], 1);
      ptx::mbar_init(&empty[i], kTcGenWarps);
    }
    for (int i = 0; i < kTcNS; ++i) {
      ptx::mbar_init(&gen[i], kTcGenWarps);
      ptx::mbar_init(&mma[i], 1);
    }
    ptx::mbar_init(drain, 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  ptx::fence_proxy_async_smem();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: A stage s at [128 s, 128 s + 128) (hi +0..63, lo +64..127), s < 3;
  // FP32 accumulators of run parity r at [384 + NP r, 384 + NP (r + 1)).
  constexpr uint32_t kAcols = kTcChunk;  // 32-bit columns of one A stage (hi and lo halves)
  constexpr uint32_t kDcol = kAcols * kTcNS;
  static_assert(kDcol + 2 * NP <= kTcCols, "tensor memory budget");
  bool failed = false;

  if (warp == kTcGenWarps) {
    // ------------------------------------------------------------ loader
    const uint32_t row_bytes = kTcChunk * 4;
    for (int i = 0; i < nchunks; ++i) {
      const int f = i % L::kNF;
      if (i >= L::kNF && !tc_wait(&empty[f], (uint32_t)(((i - L::kNF) / L::kNF) & 1), abort_flag)) {
        failed = true;
        break;
      }
      if (lane == 0) ptx::mbar_arrive_expect_tx(&full[f], row_bytes * (uint32_t)a.ns);
      __syncwarp();
      const long long base = v_begin + (long long)i * kTcChunk;
      for (int n = lane; n < a.ns; n += 32)
        ptx::bulk_g2s(fs + (size_t)f * (NP + 1) * kTcFld + (size_t)n * kTcFld,
                      a.fields + (size_t)n * a.nvox + base, row_bytes, &full[f]);
    }
  } else if (warp == kTcGenWarps + 1) {
    // ------------------------------------------------------------ MMA issuer
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, NP);
    constexpr uint32_t kSbo = (kTcChunk / 8) * 128;
    for (int i = 0; i < nchunks; ++i) {
      const int s = i % kTcNS;
      if (!tc_wait(&gen[s], (uint32_t)((i / kTcNS) & 1), abort_flag)) {
        failed = true;
        break;
      }
      ptx::tc_fence_after();
      if (lane == 0) {
        const int run = i / kTcRun;
        const bool first = (i % kTcRun) == 0;
        const uint32_t dcol = tmem + kDcol + (uint32_t)(NP * (run & 1));
        const uint32_t bhi = ptx::smem_u32(bs + (size_t)(2 * s + 0) * L::kBPart);
        const uint32_t blo = ptx::smem_u32(bs + (size_t)(2 * s + 1) * L::kBPart);
#pragma unroll
        for (int ks = 0; ks < kTcChunk / 16; ++ks) {
          const uint32_t ahi = tmem + (uint32_t)(kAcols * s + 8 * ks);
          const uint32_t alo = ahi + kAcols / 2;
          const uint64_t dh = ptx::smem_desc(bhi + 256u * ks, 128u, kSbo);
          const uint64_t dl = ptx::smem_desc(blo + 256u * ks, 128u, kSbo);
          ptx::mma_bf16_ts(dcol, ahi, dh, idesc, (first && ks == 0) ? 0u : 1u);
          ptx::mma_bf16_ts(dcol, ahi, dl, idesc, 1u);
          ptx::mma_bf16_ts(dcol, alo, dh, idesc, 1u);
        }
        ptx::mma_commit(&mma[s]);
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
    // padding rows compute d_0^2: their accumulator rows are never read (a D row depends only
    // on its own A row)
    const int ra = ab.x >= 0 ? ab.x : 0;
    const int rb = ab.x >= 0 ? ab.y : 0;
    constexpr int kCols = NP / 4;  // accumulator columns this thread flushes
    double acc[kCols];
#pragma unroll
    for (int j = 0; j < kCols; ++j) acc[j] = 0.0;
    auto flush = [&](int run) {
      const uint32_t dcol = kDcol + (uint32_t)(NP * (run & 1)) + (uint32_t)(kCols * sub);
#pragma unroll
      for (int j0 = 0; j0 < kCols; j0 += 8) {
        uint32_t v[8];
        ptx::tmem_ld8(tmem + lane_base + dcol + j0, v);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j0 + j] += (double)__uint_as_float(v[j]);
      }
    };
    // Hand a finished stage to the MMA warp: its tensor-memory stores have landed and its
    // shared-memory B rows are visible to the tensor core. Done one chunk late, so the store
    // latency overlaps the next chunk's arithmetic. One arrival per warp.
    auto publish = [&](int s) {
      ptx::tmem_st_wait();
      ptx::fence_proxy_async_smem();
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&gen[s]);
    };
    const int ka = ((ra >> 3) * (kTcChunk / 8)) * 128 + (ra & 7) * 16;  // core-matrix row of field a
    const int kb = ((rb >> 3) * (kTcChunk / 8)) * 128 + (rb & 7) * 16;
    for (int i = 0; i < nchunks; ++i) {
      const int f = i % L::kNF;
      const int s = i % kTcNS;
      bool ok = tc_wait(&full[f], (uint32_t)((i / L::kNF) & 1), abort_flag);
      if (ok && i >= kTcNS) ok = tc_wait(&mma[s], (uint32_t)(((i - kTcNS) / kTcNS) & 1), abort_flag);
      if (!ok) *abort_flag = 1;
      ptx::tc_fence_after();
      // The MMAs of chunk i - NS, the first chunk of run r, have completed, and with them every
      // MMA of run r - 1 (MMAs complete in issue order): read that run's accumulator now. Its
      // columns are next written by run r + 1, which starts only after chunk (r + 1) * RUN has
      // been generated, later in this loop.
      if (ok && i >= kTcRun && i % kTcRun == kTcNS) flush(i / kTcRun - 1);
      const float* fsf = fs + (size_t)f * (NP + 1) * kTcFld;
      unsigned char* bh_s = bs + (size_t)(2 * s + 0) * L::kBPart;
      unsigned char* bl_s = bs + (size_t)(2 * s + 1) * L::kBPart;
      // B operand (and the split fields the pair products are formed from): 8 field values,
      // one 16-byte core-matrix row, per thread and pass; rows >= ns are zero
#pragma unroll
      for (int rep = 0; rep < (NP + 31) / 32; ++rep) {
        const int t = tid + rep * kTcGen;
        const int n = ((t >> 7) << 3) + (t & 7);
        const int kc = (t >> 3) & 15;
        const float4 x0 = *reinterpret_cast<const float4*>(fsf + n * kTcFld + 8 * kc);
        const float4 x1 = *reinterpret_cast<const float4*>(fsf + n * kTcFld + 8 * kc + 4);
        uint4 h, l;
        ptx::split_bf16x2(ptx::f2_pack(x0.x, x0.y), h.x, l.x);
        ptx::split_bf16x2(ptx::f2_pack(x0.z, x0.w), h.y, l.y);
        ptx::split_bf16x2(ptx::f2_pack(x1.x, x1.y), h.z, l.z);
        ptx::split_bf16x2(ptx::f2_pack(x1.z, x1.w), h.w, l.w);
        const int off = (n >> 3) * (kTcChunk / 8) * 128 + kc * 128 + (n & 7) * 16;
        *reinterpret_cast<uint4*>(bh_s + off) = h;
        *reinterpret_cast<uint4*>(bl_s + off) = l;
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&empty[f]);  // the FP32 stage is no longer read
      // every B row of stage s is written; a failed wait anywhere stops all generator warps here
      if (ptx::named_barrier_or(1, kTcGen, !ok)) {
        failed = true;
        break;
      }
      // A operand: 32 pair products of this row from the bf16 splits of fields a and b
      uint32_t hv[16], lv[16];
      {
        const int kbase = (4 * sub) * 128;  // core-matrix columns of voxels [32 sub, 32 sub + 32)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const uint4 ah = *reinterpret_cast<const uint4*>(bh_s + ka + kbase + 128 * m);
          const uint4 al = *reinterpret_cast<const uint4*>(bl_s + ka + kbase + 128 * m);
          const uint4 bh = *reinterpret_cast<const uint4*>(bh_s + kb + kbase + 128 * m);
          const uint4 bl = *reinterpret_cast<const uint4*>(bl_s + kb + kbase + 128 * m);
          ptx::bf16x2_pair_product(ah.x, al.x, bh.x, bl.x, hv[4 * m + 0], lv[4 * m + 0]);
          ptx::bf16x2_pair_product(ah.y, al.y, bh.y, bl.y, hv[4 * m + 1], lv[4 * m + 1]);
          ptx::bf16x2_pair_product(ah.z, al.z, bh.z, bl.z, hv[4 * m + 2], lv[4 * m + 2]);
          ptx::bf16x2_pair_product(ah.w, al.w, bh.w, bl.w, hv[4 * m + 3], lv[4 * m + 3]);
        }
      }
      if (i > 0) publish((i - 1) % kTcNS);
      const uint32_t acol = (uint32_t)(kAcols * s + 16 * sub);
      ptx::tmem_st16(tmem + lane_base + acol, hv);
      ptx::tmem_st16(tmem + lane_base + acol + kAcols / 2, lv);
    }
    if (!failed && nchunks > 0) publish((nchunks - 1) % kTcNS);
    if (!failed && nchunks > 0) {
      const int last = nchunks - 1;
      if (tc_wait(&mma[last % kTcNS], (uint32_t)((last / kTcNS) & 1), abort_flag)) {
        ptx::tc_fence_after();
        const int last_run = last / kTcRun;
        // the previous run is still unread if the last run has fewer than NS + 1 chunks
        if (last_run >= 1 && last % kTcRun < kTcNS) flush(last_run - 1);
        flush(last_run);
      } else {
        failed = true;
      }
    }
    if (failed) ptx::tmem_st_wait();
    if (!failed) {
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

// msum[t] = scale * sum over voxel blocks of partial[y][map[t]], blocks in order.
__global__ void reduce_tc_kernel(const double* partial, int gridy, long long stride, const int* map, const int* bins,
                                 int n_out, double* msum, double scale) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_out) return;
  const long long off = map[t];
  double s = 0.0;
  for (int y = 0; y < gridy; ++y) s += partial[(long long)y * stride + off];
  msum[bins ? bins[t] : t] = scale * s;
}

}  // namespace

int tc_padded_shells(int ns) { return ns <= 32 ? 32 : 64; }

size_t tc_partial_doubles(int n_mtiles, int gridy, int np) { return (size_t)gridy * n_mtiles * 128 * np; }

bsp_status launch_contract_tc(const TcArgs& a, cudaStream_t s) {
  if (a.n_mtiles == 0) return BSP_OK;
  dim3 grid(a.n_mtiles, a.gridy);
  if (a.np == 32) {
    const int smem = TcSmem<32>::kBytes;
    BSP_CUDA(cudaFuncSetAttribute(contract_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    contract_tc_kernel<32><<<grid, kTcThreads, smem, s>>>(a);
  } else if (a.np == 64) {
    const int smem = TcSmem<64>::kBytes;
    BSP_CUDA(cudaFuncSetAttribute(contract_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    contract_tc_kernel<64><<<grid, kTcThreads, smem, s>>>(a);
  } else {
    return fail_c(BSP_ERR_NOT_SUPPORTED, "tensor-core contraction supports at most 64 shells");
  }
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

bsp_status launch_reduce_tc(const TcArgs& a, const int* map, const int* bins, int n_out, double* msum,
                            double scale, cudaStream_t s) {
  if (a.n_mtiles == 0 || n_out == 0) return BSP_OK;
  const long long stride = (long long)a.n_mtiles * 128 * a.np;
  reduce_tc_kernel<<<(n_out + 255) / 256, 256, 0, s>>>(a.partial, a.gridy, stride, map, bins, n_out, msum, scale);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

}  // namespace bsp
