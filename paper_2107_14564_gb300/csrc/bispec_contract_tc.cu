// Triple-product reduction on the tcgen05 tensor cores (BSP_MIXED_BF16X3 plans).
//
// The numerator of Eq. (2.7) for every kept bin is read off one dense contraction
//     M[(a,b), c] = sum_x P_ab(x) d_c(x),    P_ab = d_a d_b,
// a GEMM with M = pairs (128 per tile), N = shells (padded to NP), K = voxels. Both operands are
// split into bf16 high and low parts, P = Ph + Pl and d = dh + dl, and three MMAs per K step
// accumulate Ph dh + Ph dl + Pl dh in FP32 (relative error about 2^-16 per product).
//
// Per block (256 threads, one M tile of 128 pair rows, a contiguous voxel range):
//   * cp.async brings the FP32 fields of the next 64-voxel chunk into shared memory
//     (double buffered) while the current one is processed;
//   * every thread owns one pair row (its TMEM lane) and half of the chunk's voxels: it forms
//     the 32 pair products on CUDA cores, splits them and writes the bf16 A operand straight
//     into tensor memory with tcgen05.st (no shared-memory round trip);
//   * the threads also split the fields into the bf16 B operand in shared memory, laid out as
//     K-major core matrices (8 rows x 16 bytes) for a no-swizzle UMMA descriptor;
//   * one thread issues 12 MMAs per chunk (4 K steps x 3 products) into an FP32 accumulator in
//     tensor memory and commits them to an mbarrier; the next chunk is generated while they run;
//   * every 16 chunks (1024 voxels) the accumulator is read back (tcgen05.ld) into FP64
//     registers and a second accumulator takes over, so FP32 sums stay short.
// Blocks write FP64 partial sums; a second kernel adds them in a fixed order.
// Every wait is bounded: on give-up the block raises an error flag, drains and frees its TMEM.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace bsp {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcChunk = 64;                 // voxels per chunk (K of one stage)
constexpr int kTcRun = 16;                   // chunks per FP32 accumulation run
constexpr int kTcFld = kTcChunk + 4;         // padded FP32 row in shared memory (floats)
constexpr uint32_t kTcCols = 256;            // TMEM columns per block
constexpr long long kWaitLimit = 1LL << 22;  // mbarrier polls before giving up

template <int NP>
struct TcSmem {
  static constexpr int kFsBytes = 2 * NP * kTcFld * 4;            // [stage][NP][kTcFld] floats
  static constexpr int kBPart = NP * kTcChunk * 2;                // one bf16 operand part
  static constexpr int kBsOff = (kFsBytes + 1023) / 1024 * 1024;  // [stage][hi/lo][...]
  static constexpr int kBarOff = kBsOff + 4 * kBPart;
  static constexpr int kBytes = kBarOff + 64;
};

template <int NP>
__global__ void __launch_bounds__(kTcThreads, 2) contract_tc_kernel(TcArgs a) {
  using L = TcSmem<NP>;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* fs = reinterpret_cast<float*>(smem);
  unsigned char* bs = smem + L::kBsOff;
  // [0], [1]: MMAs of the chunk in stage 0 / 1 done; [2]: drain on the error path
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kBarOff + 24);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int quarter = warp & 3;  // TMEM lanes 32*quarter .. +31
  const int half = warp >> 2;    // voxels [32*half, 32*half + 32) of a chunk
  const int row = 32 * quarter + lane;
  const int mtile = blockIdx.x;
  const long long v_begin = (long long)blockIdx.y * a.vox_per_block;
  const long long v_end = min(v_begin + a.vox_per_block, a.nvox);
  const int nchunks = v_end > v_begin ? (int)((v_end - v_begin) / kTcChunk) : 0;
  const float* fields = a.fields;

  // zero the FP32 staging (rows >= ns are never loaded and must read as 0)
  for (int i = tid; i < L::kFsBytes / 16; i += kTcThreads)
    reinterpret_cast<float4*>(fs)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp == 0) {
    ptx::tmem_alloc(tmem_slot, kTcCols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    ptx::mbar_init(&bars[0], 1);
    ptx::mbar_init(&bars[1], 1);
    ptx::mbar_init(&bars[2], 1);
    ptx::fence_mbar_init();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // TMEM columns: A operand stage s at [64 s, 64 s + 64) (hi: +0..31, lo: +32..63);
  // FP32 accumulators of run parity r at [128 + NP r, 128 + NP (r + 1)).
  const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;

  const int2 ab = a.pair_ab[mtile * 128 + row];
  const bool real = ab.x >= 0;
  const int ra = real ? ab.x : 0;
  const int rb = real ? ab.y : 0;
  constexpr int kHalfN = NP / 2;
  double acc[kHalfN];
#pragma unroll
  for (int j = 0; j < kHalfN; ++j) acc[j] = 0.0;

  auto load_chunk = [&](int i, int s) {
    const long long base = v_begin + (long long)i * kTcChunk;
    constexpr int kPieces = kTcChunk / 4;  // 16-byte pieces per field row
    for (int idx = tid; idx < a.ns * kPieces; idx += kTcThreads) {
      const int n = idx / kPieces;
      const int j = idx - n * kPieces;
      ptx::cp_async16(fs + ((size_t)(s * NP + n) * kTcFld + 4 * j), fields + (size_t)n * a.nvox + base + 4 * j);
    }
    ptx::cp_async_commit();
  };

  auto flush = [&](int run) {
    const uint32_t dcol = 128u + (uint32_t)(NP * (run & 1)) + (uint32_t)(kHalfN * half);
#pragma unroll
    for (int j0 = 0; j0 < kHalfN; j0 += 16) {
      uint32_t v[16];
      ptx::tmem_ld16(tmem + lane_base + dcol + j0, v);
      ptx::tmem_ld_wait();
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j0 + j] += (double)__uint_as_float(v[j]);
    }
  };

  constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, NP);
  bool failed = false;
  if (nchunks > 0) load_chunk(0, 0);
  for (int i = 0; i < nchunks && !failed; ++i) {
    const int s = i & 1;
    if (i + 1 < nchunks) load_chunk(i + 1, s ^ 1);
    else ptx::cp_async_commit();
    bool ok = true;
    if (i >= 2) ok = ptx::mbar_wait(&bars[s], (uint32_t)(((i - 2) >> 1) & 1), kWaitLimit);
    if (ok && i > 0 && i % kTcRun == 0)
      ok = ptx::mbar_wait(&bars[(i - 1) & 1], (uint32_t)(((i - 1) >> 1) & 1), kWaitLimit);
    ptx::cp_async_wait<1>();
    if (__syncthreads_or(!ok)) { failed = true; break; }
    ptx::tc_fence_after();
    if (i > 0 && i % kTcRun == 0) flush(i / kTcRun - 1);

    const float* f = fs + (size_t)s * NP * kTcFld;
    // ---- B operand: fields split into bf16 hi / lo, K-major core matrices
    {
      unsigned char* bhi = bs + (size_t)(2 * s + 0) * L::kBPart;
      unsigned char* blo = bs + (size_t)(2 * s + 1) * L::kBPart;
#pragma unroll
      for (int rep = 0; rep < NP / 32; ++rep) {
        const int t = tid + rep * kTcThreads;
        const int n = ((t >> 6) << 3) + (t & 7);
        const int kc = (t >> 3) & 7;
        const float4 x0 = *reinterpret_cast<const float4*>(f + n * kTcFld + 8 * kc);
        const float4 x1 = *reinterpret_cast<const float4*>(f + n * kTcFld + 8 * kc + 4);
        uint4 h, l;
        h.x = ptx::pack_bf16x2(x0.x, x0.y);
        h.y = ptx::pack_bf16x2(x0.z, x0.w);
        h.z = ptx::pack_bf16x2(x1.x, x1.y);
        h.w = ptx::pack_bf16x2(x1.z, x1.w);
        l.x = ptx::pack_bf16x2(x0.x - ptx::bf16lo_to_f32(h.x), x0.y - ptx::bf16hi_to_f32(h.x));
        l.y = ptx::pack_bf16x2(x0.z - ptx::bf16lo_to_f32(h.y), x0.w - ptx::bf16hi_to_f32(h.y));
        l.z = ptx::pack_bf16x2(x1.x - ptx::bf16lo_to_f32(h.z), x1.y - ptx::bf16hi_to_f32(h.z));
        l.w = ptx::pack_bf16x2(x1.z - ptx::bf16lo_to_f32(h.w), x1.w - ptx::bf16hi_to_f32(h.w));
        const int off = (n >> 3) * (kTcChunk / 8) * 128 + kc * 128 + (n & 7) * 16;
        *reinterpret_cast<uint4*>(bhi + off) = h;
        *reinterpret_cast<uint4*>(blo + off) = l;
      }
    }
    // ---- A operand: pair products of this thread's row, split, into tensor memory
    {
      uint32_t hv[16], lv[16];
      const float* fa = f + ra * kTcFld + 32 * half;
      const float* fb = f + rb * kTcFld + 32 * half;
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float4 xa = *reinterpret_cast<const float4*>(fa + 4 * m);
        const float4 xb = *reinterpret_cast<const float4*>(fb + 4 * m);
        const float p0 = real ? xa.x * xb.x : 0.f;
        const float p1 = real ? xa.y * xb.y : 0.f;
        const float p2 = real ? xa.z * xb.z : 0.f;
        const float p3 = real ? xa.w * xb.w : 0.f;
        const uint32_t h0 = ptx::pack_bf16x2(p0, p1);
        const uint32_t h1 = ptx::pack_bf16x2(p2, p3);
        hv[2 * m] = h0;
        hv[2 * m + 1] = h1;
        lv[2 * m] = ptx::pack_bf16x2(p0 - ptx::bf16lo_to_f32(h0), p1 - ptx::bf16hi_to_f32(h0));
        lv[2 * m + 1] = ptx::pack_bf16x2(p2 - ptx::bf16lo_to_f32(h1), p3 - ptx::bf16hi_to_f32(h1));
      }
      const uint32_t acol = (uint32_t)(64 * s + 16 * half);
      ptx::tmem_st16(tmem + lane_base + acol, hv);
      ptx::tmem_st16(tmem + lane_base + acol + 32, lv);
      ptx::tmem_st_wait();
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      ptx::tc_fence_after();
      const int run = i / kTcRun;
      const bool first = (i % kTcRun) == 0;
      const uint32_t dcol = tmem + 128u + (uint32_t)(NP * (run & 1));
      const uint32_t bhi = ptx::smem_u32(bs + (size_t)(2 * s + 0) * L::kBPart);
      const uint32_t blo = ptx::smem_u32(bs + (size_t)(2 * s + 1) * L::kBPart);
      constexpr uint32_t kSbo = (kTcChunk / 8) * 128;
#pragma unroll
      for (int ks = 0; ks < kTcChunk / 16; ++ks) {
        const uint32_t ahi = tmem + (uint32_t)(64 * s + 8 * ks);
        const uint32_t alo = ahi + 32u;
        const uint64_t dh = ptx::smem_desc(bhi + 256u * ks, 128u, kSbo);
        const uint64_t dl = ptx::smem_desc(blo + 256u * ks, 128u, kSbo);
        ptx::mma_bf16_ts(dcol, ahi, dh, idesc, (first && ks == 0) ? 0u : 1u);
        ptx::mma_bf16_ts(dcol, ahi, dl, idesc, 1u);
        ptx::mma_bf16_ts(dcol, alo, dh, idesc, 1u);
      }
      ptx::mma_commit(&bars[s]);
    }
  }
  if (!failed && nchunks > 0) {
    const int last = nchunks - 1;
    const bool ok = ptx::mbar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1), kWaitLimit);
    if (__syncthreads_or(!ok)) {
      failed = true;
    } else {
      ptx::tc_fence_after();
      flush(last / kTcRun);
    }
  }
  ptx::cp_async_wait<0>();
  if (failed) {
    // let the MMAs already issued drain (bounded) before the tensor memory is released
    if (tid == 0) {
      atomicExch(a.error, 1);
      ptx::mma_commit(&bars[2]);
    }
    ptx::mbar_wait(&bars[2], 0u, kWaitLimit);
  } else {
    double* out = a.partial + (((size_t)blockIdx.y * a.n_mtiles + mtile) * 128 + row) * NP + kHalfN * half;
#pragma unroll
    for (int j = 0; j < kHalfN; ++j) out[j] = acc[j];
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, kTcCols);
  }
}

// msum[t] = sum over voxel blocks of partial[y][map[t]], blocks in order.
__global__ void reduce_tc_kernel(const double* partial, int gridy, long long stride, const int* map, int n_out,
                                 double* msum) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_out) return;
  const long long off = map[t];
  double s = 0.0;
  for (int y = 0; y < gridy; ++y) s += partial[(long long)y * stride + off];
  msum[t] = s;
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

bsp_status launch_reduce_tc(const TcArgs& a, const int* map, int n_out, double* msum, cudaStream_t s) {
  if (a.n_mtiles == 0 || n_out == 0) return BSP_OK;
  const long long stride = (long long)a.n_mtiles * 128 * a.np;
  reduce_tc_kernel<<<(n_out + 255) / 256, 256, 0, s>>>(a.partial, a.gridy, stride, map, n_out, msum);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

}  // namespace bsp
