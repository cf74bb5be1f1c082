// Triple-product reduction on CUDA cores and the final normalisation.
//
// msum[t] = sum_x d_a(x) d_b(x) d_c(x) for every kept bin t = (a, b, c) (numerator of Eq. (2.7);
// with counting fields, the T_abc of Eq. (2.10)). The bins are grouped as
// M[(a,b), c] = sum_x (d_a d_b)(x) d_c(x): a tile owns up to 4 pairs (a, b) and 4 consecutive
// c, i.e. 16 outputs held in registers by one thread. A block walks a contiguous voxel range in
// chunks staged in shared memory (all shells of the chunk), so every field value read from
// HBM serves every tile of the block; the next chunk is copied in with cp.async into a second
// buffer while the current one is used. FP32 plans accumulate in FP32 over kFlushChunks chunks
// and then add into FP64; FP64 plans accumulate in FP64. Blocks write FP64 partial sums,
// which a second kernel adds in a fixed order (deterministic results).
#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace bsp {

constexpr int kChunk = 64;         // voxels per shared-memory chunk
constexpr int kContractThreads = 256;
constexpr int kFlushChunks = 16;   // FP32 run length: 1024 voxels

// Two neighbouring voxels of one field, read from shared memory in one 8-byte (FP32) or
// 16-byte (FP64) load.
template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };
// Row stride of a staged chunk: even, so voxel pairs are aligned; 66 words puts field n's pair
// (v, v + 1) on the bank pair (n + v / 2) mod 16.
constexpr int kChunkLd = kChunk + 2;

template <typename T>
__global__ void __launch_bounds__(kContractThreads)
contract_simt_kernel(ContractArgs a, long long vox_per_block) {
  using T2 = typename Pair2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* dsm0 = reinterpret_cast<T*>(smem_raw);  // two chunks [ns][kChunkLd]
  constexpr int LD = kChunkLd;
  const int chunk_elems = a.ns * LD;
  const T* fields = static_cast<const T*>(a.fields);
  const int tile = blockIdx.y * kContractThreads + threadIdx.x;
  const bool active = tile < a.ntiles;
  int ia[4], ib[4], c0 = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) { ia[i] = 0; ib[i] = 0; }
  if (active) {
    const Tile t = a.tiles[tile];
    c0 = t.c0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int p = t.p0 + (i < t.np ? i : 0);
      const int2 ab = a.pairs[p];
      ia[i] = ab.x;
      ib[i] = ab.y;
    }
  }
  int ic[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) ic[j] = min(c0 + j, a.ns - 1);

  double acc64[16];
  T acc[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) { acc64[k] = 0.0; acc[k] = T(0); }

  const long long v_begin = (long long)blockIdx.x * vox_per_block;
  const long long v_end = min(v_begin + vox_per_block, a.nvox);
  // copy the chunk at vb into dst (zeros past v_end), one commit group
  auto stage = [&](long long vb, T* dst) {
    for (int i = threadIdx.x; i < a.ns * kChunk; i += kContractThreads) {
      const int n = i / kChunk;
      const int v = i - n * kChunk;
      const long long gv = vb + v;
      const bool in = gv < v_end;
      ptx::cp_async_zfill<(int)sizeof(T)>(dst + n * LD + v, in ? fields + (long long)n * a.nvox + gv : fields,
                                          in ? (uint32_t)sizeof(T) : 0u);
    }
    ptx::cp_async_commit();
  };
  if (v_begin < v_end) stage(v_begin, dsm0);
  int run = 0, k = 0;
  for (long long vb = v_begin; vb < v_end; vb += kChunk, ++k) {
    const T* dsm = dsm0 + (size_t)(k & 1) * chunk_elems;
    if (vb + kChunk < v_end) {
      stage(vb + kChunk, dsm0 + (size_t)((k + 1) & 1) * chunk_elems);
      ptx::cp_async_wait<1>();  // this chunk's copies (issued one iteration earlier) have landed
    } else {
      ptx::cp_async_wait<0>();
    }
    __syncthreads();
    if (active) {
#pragma unroll 2
      for (int v = 0; v < kChunk; v += 2) {  // voxels v and v + 1, added in that order
        T2 p[4], d[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T2 x = *reinterpret_cast<const T2*>(dsm + ia[i] * LD + v);
          const T2 y = *reinterpret_cast<const T2*>(dsm + ib[i] * LD + v);
          p[i].x = x.x * y.x;
          p[i].y = x.y * y.y;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) d[j] = *reinterpret_cast<const T2*>(dsm + ic[j] * LD + v);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i * 4 + j] = fma(p[i].x, d[j].x, acc[i * 4 + j]);
            acc[i * 4 + j] = fma(p[i].y, d[j].y, acc[i * 4 + j]);
          }
      }
      if (++run == kFlushChunks) {
        run = 0;
#pragma unroll
        for (int q = 0; q < 16; ++q) { acc64[q] += (double)acc[q]; acc[q] = T(0); }
      }
    }
    __syncthreads();  // every thread is done with this buffer before the next copy into it
  }
  if (active) {  // partial[(tile * 16 + k) * gridx + block]: an output's block sums are contiguous
    double* out = a.partial + (long long)tile * 16 * a.gridx + blockIdx.x;
#pragma unroll
    for (int k = 0; k < 16; ++k) out[(long long)k * a.gridx] = acc64[k] + (double)acc[k];
  }
}

// msum[map[tile][k]] = scale * sum over blocks of partial[tile][k][block], in a fixed order
// (added to msum when accumulating x-slabs).
// One warp per (tile, entry): lane l adds the block sums b = l, l + 32, ... (contiguous loads
// across the warp), then the lanes' sums are added by a fixed shuffle tree.
__global__ void reduce_partials_kernel(ContractArgs a) {
  const int idx = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= a.ntiles * 16) return;  // warp-uniform
  const int dst = a.tile_map[idx];
  if (dst < 0) return;  // warp-uniform
  const double* src = a.partial + (long long)idx * a.gridx;
  double s = 0.0;
  for (int b = lane; b < a.gridx; b += 32) s += src[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) a.msum[dst] = a.accumulate ? a.msum[dst] + a.scale * s : a.scale * s;
}

template <typename T>
bsp_status launch_contract_simt(const ContractArgs& a, cudaStream_t s) {
  if (a.ntiles == 0) return BSP_OK;
  const long long chunks = (a.nvox + kChunk - 1) / kChunk;
  const long long per_block_chunks = (chunks + a.gridx - 1) / a.gridx;
  const long long vpb = per_block_chunks * kChunk;
  dim3 grid(a.gridx, (a.ntiles + kContractThreads - 1) / kContractThreads);
  const size_t smem = 2 * (size_t)a.ns * kChunkLd * sizeof(T);
  BSP_CUDA(cudaFuncSetAttribute(contract_simt_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  contract_simt_kernel<T><<<grid, kContractThreads, smem, s>>>(a, vpb);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

bsp_status launch_reduce_partials(const ContractArgs& a, cudaStream_t s) {
  const long long n = (long long)a.ntiles * 16 * 32;  // one warp per entry
  if (n == 0) return BSP_OK;
  reduce_partials_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

// ---------------------------------------------------------------- product fields (order 4)
template <typename T>
__global__ void pair_fields_kernel(const T* __restrict__ f, long long nvox, const int2* __restrict__ pairs, int np,
                                   T* __restrict__ out) {
  const long long total = nvox * np;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / nvox);
    const long long v = i - (long long)j * nvox;
    const int2 ab = pairs[j];
    out[i] = f[(long long)ab.x * nvox + v] * f[(long long)ab.y * nvox + v];
  }
}

template <typename T>
bsp_status launch_pair_fields(const void* f, long long nvox, const int2* pairs, int np, void* out, int n_sm,
                              cudaStream_t s) {
  if (np == 0 || nvox == 0) return BSP_OK;
  const long long need = (nvox * np + 255) / 256;
  const long long blocks = std::min<long long>(need, 8LL * std::max(n_sm, 1));
  pair_fields_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const T*>(f), nvox, pairs, np,
                                                         static_cast<T*>(out));
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template bsp_status launch_pair_fields<float>(const void*, long long, const int2*, int, void*, int, cudaStream_t);
template bsp_status launch_pair_fields<double>(const void*, long long, const int2*, int, void*, int, cudaStream_t);
template bsp_status launch_contract_simt<float>(const ContractArgs&, cudaStream_t);
template bsp_status launch_contract_simt<double>(const ContractArgs&, cudaStream_t);

// ---------------------------------------------------------------- level fields
// dst[j][x][y][z] = src[shells[j]][t x][t y][t z]: the fields of a coarser level sampled from the
// evaluation grid (side S) with stride t.
template <typename T>
__global__ void decimate_kernel(const T* __restrict__ src, int S, const int* __restrict__ shells, int nsh,
                                T* __restrict__ dst, int g, int t) {
  const long long per = (long long)g * g * g;
  const long long total = per * nsh;
  const long long plane = (long long)S * S;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(i / per);
    const long long v = i - (long long)j * per;
    const int x = (int)(v / ((long long)g * g));
    const int y = (int)((v / g) % g);
    const int z = (int)(v % g);
    dst[i] = src[(long long)shells[j] * plane * S + ((long long)x * t * S + (long long)y * t) * S + (long long)z * t];
  }
}

template <typename T>
bsp_status launch_decimate(const void* src, int S, const int* shells, int nsh, void* dst, int g, int t, int n_sm,
                           cudaStream_t s) {
  const long long total = (long long)g * g * g * nsh;
  if (total == 0) return BSP_OK;
  long long blocks = std::min<long long>((total + 255) / 256, 16LL * n_sm);
  decimate_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const T*>(src), S, shells, nsh, static_cast<T*>(dst),
                                                     g, t);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}
template bsp_status launch_decimate<float>(const void*, int, const int*, int, void*, int, int, int, cudaStream_t);
template bsp_status launch_decimate<double>(const void*, int, const int*, int, void*, int, int, int, cudaStream_t);
template bsp_status launch_decimate<uint16_t>(const void*, int, const int*, int, void*, int, int, int, cudaStream_t);

// ---------------------------------------------------------------- finalize
// b_trip[t] = norm msum[t] / tsum[t]                     (Eq. (2.7) with Eq. (2.10))
// b_grid[cell] = norm sum msum / sum tsum over the cell's bins, NaN if it has none.
__global__ void finalize_kernel(FinalizeArgs a) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < a.n_trip) a.b_trip[idx] = a.norm * a.msum[idx] / a.tsum[idx];
  if (a.b_grid != nullptr && idx < a.n_cells) {
    const int lo = a.cell_ptr[idx], hi = a.cell_ptr[idx + 1];
    if (lo == hi) {
      a.b_grid[idx] = __longlong_as_double(0x7ff8000000000000ULL);
    } else {
      double num = 0.0, den = 0.0;
      for (int i = lo; i < hi; ++i) {
        const int t = a.cell_idx[i];
        num += a.msum[t];
        den += a.tsum[t];
      }
      a.b_grid[idx] = a.norm * num / den;
    }
  }
}

bsp_status launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
  const int n = a.n_trip > a.n_cells ? a.n_trip : a.n_cells;
  if (n == 0) return BSP_OK;
  finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(a);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

}  // namespace bsp
