// Kernels of the adjoint (gradient) of the estimator with respect to delta(x).
//
// For an upstream gradient g_t = dL/dB_t and c_t = V_c^3 / (V T_t) (Eq. (2.7) with Eq. (2.10)),
// B_t = c_t sum_x d_a d_b d_c is trilinear in the shell fields, so
//   dL/d delta(y) = sum_k [ sum_n S_n(k) K(k) G^_n(k) ] e^{+i k.y},
//   G_n(x) = sum_t g_t c_t sum_{positions of n in t} (product of the other two fields),
// with G^_n the forward DFT of G_n over the grid and K the optional Kaiser factor (Eq. (3.4)).
// G_n is formed on the evaluation grid as a small dense product G[n](x) = sum_p W[p][n] P_p(x)
// over pairs p = (a, b), a >= b, with P_p = d_a d_b and W[p][n] collecting the g_t c_t of every
// bin position whose other two shells are p.
#include "common.cuh"

namespace bsp {
namespace {

constexpr int kAdjThreads = 128;

// W[e] = sum over the bins listed for entry e of g_t c_t, in list order (deterministic).
__global__ void build_w_kernel(const double* g, const double* cnorm, const int* ptr, const int* idx, int n_entries,
                               float* W) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_entries) return;
  double s = 0.0;
  for (int i = ptr[e]; i < ptr[e + 1]; ++i) s += g[idx[i]] * cnorm[idx[i]];
  W[e] = (float)s;
}

// G[n][v] = sum_p W[p][n] d_a(v) d_b(v); VPT voxels per thread, NP padded shells per W row.
template <int NP, int VPT>
__global__ void __launch_bounds__(kAdjThreads) adjoint_products_kernel(const float* __restrict__ fields, long long nvox,
                                                                       int ns, const int2* __restrict__ pairs,
                                                                       int npairs, const float* __restrict__ W,
                                                                       float* __restrict__ G) {
  constexpr int VB = kAdjThreads * VPT;  // voxels per block pass
  constexpr int LD = VB + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* fs = reinterpret_cast<float*>(smem_raw);  // [ns][LD]
  const int t = threadIdx.x;
  for (long long base = (long long)blockIdx.x * VB; base < nvox; base += (long long)gridDim.x * VB) {
    __syncthreads();
    for (int i = t; i < ns * VB; i += kAdjThreads) {
      const int n = i / VB;
      const int v = i - n * VB;
      fs[n * LD + v] = base + v < nvox ? fields[(long long)n * nvox + base + v] : 0.f;
    }
    __syncthreads();
    float acc[VPT][NP];
#pragma unroll
    for (int j = 0; j < VPT; ++j)
#pragma unroll
      for (int n = 0; n < NP; ++n) acc[j][n] = 0.f;
    for (int p = 0; p < npairs; ++p) {
      const int2 ab = pairs[p];
      float prod[VPT];
#pragma unroll
      for (int j = 0; j < VPT; ++j) prod[j] = fs[ab.x * LD + t + j * kAdjThreads] * fs[ab.y * LD + t + j * kAdjThreads];
      const float4* wrow = reinterpret_cast<const float4*>(W + (size_t)p * NP);
#pragma unroll
      for (int n4 = 0; n4 < NP / 4; ++n4) {
        const float4 w = __ldg(wrow + n4);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          acc[j][4 * n4 + 0] = fmaf(w.x, prod[j], acc[j][4 * n4 + 0]);
          acc[j][4 * n4 + 1] = fmaf(w.y, prod[j], acc[j][4 * n4 + 1]);
          acc[j][4 * n4 + 2] = fmaf(w.z, prod[j], acc[j][4 * n4 + 2]);
          acc[j][4 * n4 + 3] = fmaf(w.w, prod[j], acc[j][4 * n4 + 3]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const long long v = base + t + j * kAdjThreads;
      if (v < nvox) {
#pragma unroll
        for (int n = 0; n < NP; ++n)
          if (n < ns) G[(long long)n * nvox + v] = acc[j][n];
      }
    }
  }
}

}  // namespace

bsp_status launch_build_w(const double* g, const double* cnorm, const int* ptr, const int* idx, int n_entries,
                          float* W, cudaStream_t s) {
  if (n_entries == 0) return BSP_OK;
  build_w_kernel<<<(n_entries + 255) / 256, 256, 0, s>>>(g, cnorm, ptr, idx, n_entries, W);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

bsp_status launch_adjoint_products(const float* fields, long long nvox, int ns, int np, const int2* pairs,
                                   int npairs, const float* W, float* G, int n_sm, cudaStream_t s) {
  if (np == 32) {
    constexpr int VB = kAdjThreads * 2;
    const size_t smem = (size_t)ns * (VB + 1) * sizeof(float);
    BSP_CUDA(cudaFuncSetAttribute(adjoint_products_kernel<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    long long blocks = std::min<long long>((nvox + VB - 1) / VB, 8LL * n_sm);
    adjoint_products_kernel<32, 2><<<(unsigned)blocks, kAdjThreads, smem, s>>>(fields, nvox, ns, pairs, npairs, W, G);
  } else if (np == 64) {
    constexpr int VB = kAdjThreads;
    const size_t smem = (size_t)ns * (VB + 1) * sizeof(float);
    BSP_CUDA(cudaFuncSetAttribute(adjoint_products_kernel<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    long long blocks = std::min<long long>((nvox + VB - 1) / VB, 8LL * n_sm);
    adjoint_products_kernel<64, 1><<<(unsigned)blocks, kAdjThreads, smem, s>>>(fields, nvox, ns, pairs, npairs, W, G);
  } else {
    return fail_c(BSP_ERR_NOT_SUPPORTED, "gradient: at most 64 shells");
  }
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

}  // namespace bsp
