// Shell-pruned inverse FFT passes that turn a half spectrum into real shell fields,
// d_n(x) = sum_{k in shell n} F(k) e^{+i k.x}  (Eq. (2.8); with a unit input, Eq. (2.11)).
//
// The 3D inverse transform of one shell is done as three batched 1D passes over a spectrum
// whose support is the ball |m| < r_n (r_n <= Ng/3 + 1 by the cap after Eq. (2.12)):
//   X pass: for every (ky, kz >= 0) line that meets the ball, gather the masked line along kx
//           (only |kx| < r_n can be non-zero), transform along x -> G1[x][ky][kz]
//   Y pass: for every (x, kz < r_n) gather along ky (only |ky| < r_n), transform -> G2[x][y][kz]
//   Z pass: for every (x, y) a complex-to-real transform of the r_n leading kz values -> d_n
// Empty lines are never read or transformed. Each block holds a batch of lines in shared
// memory and runs an in-place mixed-radix Stockham transform (radices 8, 4, 2, 3) on them;
// global loads and stores run along the contiguous kz (X, Y) or z (Z) axis.
#include "common.cuh"
#include "fft_radix.cuh"

namespace bsp {

// ---------------------------------------------------------------- one Stockham stage
// Lines of length N sit at buf + l * lstride. Stage with radix R combines sub-transforms of
// length Ns: butterfly j reads x[j + r N/R], twiddles by w^{r k} (k = j mod Ns,
// w = exp(+2 pi i / (Ns R))), and writes y[(j - k) R + k + r Ns]. In place: every thread
// first loads, a barrier, then every thread stores.
template <typename T, int R>
__device__ __forceinline__ void fft_stage(cplx<T>* buf, int nlines, int lstride, int N, int Ns,
                                          const cplx<T>* tw, int twstride) {
  using C = cplx<T>;
  constexpr int E = FftElems<T>::value;
  constexpr int NB = (E + R - 1) / R;
  const int nbf = N / R;
  const int total = nlines * nbf;
  const int tunit = (N / (Ns * R)) * twstride;
  C v[NB][R];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * kFftThreads;
    if (b < total) {
      const int l = b / nbf;
      const int j = b - l * nbf;
      const C* line = buf + l * lstride;
      const int k = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C x = line[j + r * nbf];
        if (r > 0) x = c_mul(x, tw[r * k * tunit]);
        v[i][r] = x;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = threadIdx.x + i * kFftThreads;
    if (b < total) {
      Dft<C, R>::run(v[i]);
      const int l = b / nbf;
      const int j = b - l * nbf;
      C* line = buf + l * lstride;
      const int k = j % Ns;
      const int d = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) line[d + r * Ns] = v[i][r];
    }
  }
  __syncthreads();
}

// Unnormalised inverse FFT of nlines lines in shared memory. tw[j * twstride] = exp(2 pi i j/N).
template <typename T>
__device__ void fft_lines(cplx<T>* buf, int nlines, int lstride, const FftStages& st,
                          const cplx<T>* tw, int twstride) {
  int ns = 1;
  for (int s = 0; s < st.nst; ++s) {
    const int R = st.radix[s];
    if (R == 8) fft_stage<T, 8>(buf, nlines, lstride, st.n, ns, tw, twstride);
    else if (R == 4) fft_stage<T, 4>(buf, nlines, lstride, st.n, ns, tw, twstride);
    else if (R == 2) fft_stage<T, 2>(buf, nlines, lstride, st.n, ns, tw, twstride);
    else fft_stage<T, 3>(buf, nlines, lstride, st.n, ns, tw, twstride);
    ns *= R;
  }
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* tws, const void* tw, int ng) {
  const cplx<T>* src = static_cast<const cplx<T>*>(tw);
  for (int i = threadIdx.x; i < ng; i += blockDim.x) tws[i] = src[i];
}

// ---------------------------------------------------------------- X pass
template <typename T>
__global__ void __launch_bounds__(kFftThreads) xpass_kernel(PassArgs a, int max_lines) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ng = a.ng;   // input spectrum grid
  const int S = a.ngs;   // evaluation grid: line length
  C* tws = buf + (size_t)max_lines * S;
  const Item it = a.items[blockIdx.x];
  const ShellGeom g = a.geom[it.n];
  const int nl = it.cnt;
  load_twiddles<T>(tws, a.tw, S);
  for (int i = threadIdx.x; i < nl * S; i += blockDim.x) buf[i] = c_make<C>(T(0), T(0));
  __syncthreads();
  const int r = g.r;
  const int w = 2 * r - 1;
  const int ky = it.u;
  const int hz = ng / 2 + 1;
  const int iy = ky < 0 ? ky + ng : ky;
  const C* spec = static_cast<const C*>(a.spec);
  for (int idx = threadIdx.x; idx < w * nl; idx += blockDim.x) {
    const int kzl = idx % nl;
    const int mx = idx / nl - (r - 1);
    const int kz = it.v0 + kzl;
    const int q = mx * mx + ky * ky + kz * kz;
    if (q >= g.qlo && q < g.qhi) {
      const int ix = mx < 0 ? mx + ng : mx;
      C val = spec ? spec[((long long)ix * ng + iy) * hz + kz]
                   : c_make<C>(a.kweight ? T(sqrt((double)q)) : T(1), T(0));
      if (a.rsd) {
        const T fac = T(1.0 + a.beta * (double)(kz * kz) / (double)q);
        val = c_scale(val, fac);
      }
      buf[kzl * S + (mx < 0 ? mx + S : mx)] = val;
    }
  }
  __syncthreads();
  fft_lines<T>(buf, nl, S, a.st, tws, 1);
  const int jy = ky + r - 1;
  C* g1 = static_cast<C*>(a.g1) + g.g1_off;
  for (int idx = threadIdx.x; idx < S * nl; idx += blockDim.x) {
    const int kzl = idx % nl;
    const int x = idx / nl;
    g1[((long long)x * w + jy) * r + it.v0 + kzl] = buf[kzl * S + x];
  }
}

// ---------------------------------------------------------------- Y pass
template <typename T>
__global__ void __launch_bounds__(kFftThreads) ypass_kernel(PassArgs a, int max_lines) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ng = a.ngs;  // evaluation grid
  C* tws = buf + (size_t)max_lines * ng;
  const Item it = a.items[blockIdx.x];
  const ShellGeom g = a.geom[it.n];
  const int nl = it.cnt;
  load_twiddles<T>(tws, a.tw, ng);
  for (int i = threadIdx.x; i < nl * ng; i += blockDim.x) buf[i] = c_make<C>(T(0), T(0));
  __syncthreads();
  const int r = g.r;
  const int w = 2 * r - 1;
  const int x = it.u;
  const C* g1 = static_cast<const C*>(a.g1) + g.g1_off;
  for (int idx = threadIdx.x; idx < w * nl; idx += blockDim.x) {
    const int kzl = idx % nl;
    const int jy = idx / nl;
    const int ky = jy - (r - 1);
    const int kz = it.v0 + kzl;
    if (ky * ky + kz * kz < g.qhi) {
      const int iy = ky < 0 ? ky + ng : ky;
      buf[kzl * ng + iy] = g1[((long long)x * w + jy) * r + kz];
    }
  }
  __syncthreads();
  fft_lines<T>(buf, nl, ng, a.st, tws, 1);
  C* g2 = static_cast<C*>(a.g2) + g.g2_off;
  for (int idx = threadIdx.x; idx < ng * nl; idx += blockDim.x) {
    const int kzl = idx % nl;
    const int y = idx / nl;
    g2[((long long)x * ng + y) * r + it.v0 + kzl] = buf[kzl * ng + y];
  }
}

// ---------------------------------------------------------------- Z pass (complex to real)
// A real line x[0..N) with Hermitian spectrum X[0..N/2] is obtained from one complex inverse
// transform of length M = N/2: with W = exp(2 pi i / N),
//   Z[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k]) W^k,   z = IDFT_M(Z),
// and z[n] = x[2n] + i x[2n+1]. X[M] (the Nyquist plane) is never inside a shell.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) zpass_kernel(PassArgs a, int max_lines) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ng = a.ngs;  // evaluation grid
  const int M = ng / 2;
  C* tws = buf + (size_t)max_lines * M;
  const Item it = a.items[blockIdx.x];
  const ShellGeom g = a.geom[it.n];
  const int nl = it.cnt;
  load_twiddles<T>(tws, a.tw, ng);
  for (int i = threadIdx.x; i < nl * M; i += blockDim.x) buf[i] = c_make<C>(T(0), T(0));
  __syncthreads();
  const int r = g.r;
  const int x = it.u;
  const C* g2 = static_cast<const C*>(a.g2) + g.g2_off + ((long long)x * ng + it.v0) * r;
  for (int idx = threadIdx.x; idx < r * nl; idx += blockDim.x) {
    const int l = idx / r;
    const int k = idx - l * r;
    buf[l * M + k] = g2[idx];
  }
  __syncthreads();
  const int half = M / 2 + 1;
  for (int idx = threadIdx.x; idx < nl * half; idx += blockDim.x) {
    const int l = idx / half;
    const int k = idx - l * half;
    C* line = buf + l * M;
    const C xk = line[k];
    const C xmk = k == 0 ? c_make<C>(T(0), T(0)) : line[M - k];
    const C zk = c_add(c_add(xk, c_conj(xmk)), c_muli(c_mul(c_sub(xk, c_conj(xmk)), tws[k])));
    if (k > 0 && M - k != k) {
      const C zmk = c_add(c_add(xmk, c_conj(xk)), c_muli(c_mul(c_sub(xmk, c_conj(xk)), tws[M - k])));
      line[M - k] = zmk;
    }
    line[k] = zk;
  }
  __syncthreads();
  fft_lines<T>(buf, nl, M, a.st, tws, 2);
  const int nx = a.slab_nx ? a.slab_nx : ng;  // x-planes of each shell in the output
  const int x0 = a.slab_nx ? a.slab_x0 : 0;
  C* out = reinterpret_cast<C*>(static_cast<T*>(a.fields) + (long long)it.n * nx * ng * ng +
                                ((long long)(x - x0) * ng + it.v0) * ng);
  for (int idx = threadIdx.x; idx < nl * M; idx += blockDim.x) out[idx] = buf[idx];
}

// ---------------------------------------------------------------- 2D rings: X pass
// Item (n, -, v0, cnt): the k_y lines v0 .. v0 + cnt - 1 of ring n (|k_y| < r, k_y >= 0 on the
// halved axis). Gathers the ring's modes along k_x (|k_x| < r) from the 2D half spectrum
// [ng][ng/2 + 1], transforms along x on the evaluation grid (length ngs) and writes
// G[g1_off + x r + k_y], the rows the C2R along y then reads.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) ring_xpass_kernel(PassArgs a, int max_lines) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int ng = a.ng;
  const int S = a.ngs;
  C* tws = buf + (size_t)max_lines * S;
  const Item it = a.items[blockIdx.x];
  const ShellGeom g = a.geom[it.n];
  const int nl = it.cnt;
  load_twiddles<T>(tws, a.tw, S);
  for (int i = threadIdx.x; i < nl * S; i += blockDim.x) buf[i] = c_make<C>(T(0), T(0));
  __syncthreads();
  const int r = g.r;
  const int w = 2 * r - 1;
  const int hy = ng / 2 + 1;
  const C* spec = static_cast<const C*>(a.spec);
  for (int idx = threadIdx.x; idx < w * nl; idx += blockDim.x) {
    const int l = idx % nl;
    const int mx = idx / nl - (r - 1);
    const int ky = it.v0 + l;
    const int q = mx * mx + ky * ky;
    if (q >= g.qlo && q < g.qhi) {
      const int ix = mx < 0 ? mx + ng : mx;
      buf[l * S + (mx < 0 ? mx + S : mx)] = spec ? spec[(long long)ix * hy + ky] : c_make<C>(T(1), T(0));
    }
  }
  __syncthreads();
  fft_lines<T>(buf, nl, S, a.st, tws, 1);
  C* out = static_cast<C*>(a.g1) + g.g1_off;
  for (int idx = threadIdx.x; idx < S * nl; idx += blockDim.x) {
    const int l = idx % nl;
    const int x = idx / nl;
    out[(long long)x * r + it.v0 + l] = buf[l * S + x];
  }
}

// ---------------------------------------------------------------- twiddles
template <typename T>
__global__ void twiddle_kernel(cplx<T>* tw, int ng) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ng) {
    double s, c;
    sincospi(2.0 * (double)j / (double)ng, &s, &c);
    tw[j] = c_make<cplx<T>>(T(c), T(s));
  }
}

// ---------------------------------------------------------------- launchers
template <typename T>
static size_t pass_smem(int lines, int len, int ng) {
  return ((size_t)lines * len + ng) * sizeof(cplx<T>);
}

template <typename T, typename K>
static bsp_status launch_pass(K kernel, const PassArgs& a, int n_items, int lines, int len,
                              cudaStream_t s) {
  if (n_items == 0) return BSP_OK;
  const size_t smem = pass_smem<T>(lines, len, a.ngs);
  BSP_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kernel<<<n_items, kFftThreads, smem, s>>>(a, lines);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template <typename T>
bsp_status launch_xpass(const PassArgs& a, int n_items, int lines, cudaStream_t s) {
  return launch_pass<T>(xpass_kernel<T>, a, n_items, lines, a.ngs, s);
}
template <typename T>
bsp_status launch_ypass(const PassArgs& a, int n_items, int lines, cudaStream_t s) {
  return launch_pass<T>(ypass_kernel<T>, a, n_items, lines, a.ngs, s);
}
template <typename T>
bsp_status launch_zpass(const PassArgs& a, int n_items, int lines, cudaStream_t s) {
  return launch_pass<T>(zpass_kernel<T>, a, n_items, lines, a.ngs / 2, s);
}
template <typename T>
bsp_status launch_ring_xpass(const PassArgs& a, int n_items, int lines, cudaStream_t s) {
  return launch_pass<T>(ring_xpass_kernel<T>, a, n_items, lines, a.ngs, s);
}
template <typename T>
bsp_status launch_twiddles(void* tw, int ng, cudaStream_t s) {
  twiddle_kernel<T><<<(ng + 255) / 256, 256, 0, s>>>(static_cast<cplx<T>*>(tw), ng);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template bsp_status launch_ring_xpass<float>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_ring_xpass<double>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_xpass<float>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_xpass<double>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_ypass<float>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_ypass<double>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_zpass<float>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_zpass<double>(const PassArgs&, int, int, cudaStream_t);
template bsp_status launch_twiddles<float>(void*, int, cudaStream_t);
template bsp_status launch_twiddles<double>(void*, int, cudaStream_t);

}  // namespace bsp
