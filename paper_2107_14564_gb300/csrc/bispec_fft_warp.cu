// Warp-per-line shell FFT passes for FP32 plans whose grid side is a power of two (128..1024).
//
// Same three passes as the generic kernels (X and Y: C2C of the lines that meet each shell's
// ball; Z: C2R of the r_n leading k_z values into the real shell field d_n, Eq. (2.8)), but every
// line is transformed by one warp with all index arithmetic fixed at compile time:
//   * a lane holds N/32 points of the line in registers; a Stockham stage of radix R runs
//     N/(32 R) butterflies per lane, and between stages the warp exchanges its points through
//     its own padded shared-memory buffer (one __syncwarp, no block barrier);
//   * the first stage reads x[j + r N/R] and the last writes y[j + r N/R], j = lane + 32 b, so a
//     warp's global loads and stores are contiguous along the line;
//   * X and Y passes stage a [2r_n - 1][16] tile of their input (16 lines, contiguous along k_z)
//     and a [N][16] tile of their output in shared memory, so global traffic stays coalesced
//     even though their lines run along the slow axes;
//   * the Z pass forms the half-length input Z[k] = (X[k] + conj X[M-k]) + i (X[k] - conj X[M-k])
//     W^k directly from global memory and writes z[n] = x[2n] + i x[2n+1] straight to the field.
#include "common.cuh"
#include "fft_radix.cuh"
#include "tc_ptx.cuh"

#include <math.h>

#include <vector>

namespace bsp {
namespace {

constexpr int kLines = 8;           // lines per X/Y block
constexpr int kZThreads = 256;      // 8 warps, one line at a time each
constexpr int kTileLd = kLines + 1; // padded tile row (complex)

// Placement of point i in the per-line exchange buffers, chosen per length and radix list by
// counting the shared-memory wavefronts of every stage's load and store pattern (64-bit accesses,
// two half-warp phases): length 384 permutes i by i XOR ((i >> 3) & 15) (no extra space), 96 is
// unpadded, the others get one spare slot every 2^shift points (shift 2 for 64, else 4).
template <int N> struct Pad {
  static constexpr bool kXor = N == 384;
  static constexpr int shift = (kXor || N == 96) ? 0 : (N == 64 ? 2 : 4);
};
template <int N> __device__ __forceinline__ int padn(int i) {
  if constexpr (Pad<N>::kXor) return i ^ ((i >> 3) & 15);
  return Pad<N>::shift ? i + (i >> Pad<N>::shift) : i;
}
template <int N> __host__ __device__ constexpr int pad_len() { return Pad<N>::shift ? N + (N >> Pad<N>::shift) : N; }
// Line stride of the X/Y buffers: 2 mod 16 complex, so the transposed read-out (8 lines x 2
// consecutive points per half-warp) hits 16 distinct bank pairs.
template <int N> __host__ __device__ constexpr int line_ld() { return pad_len<N>() + ((18 - pad_len<N>() % 16) % 16); }

// Radix list and lanes per line of each supported length: every radix divides the points per
// lane E = N / LPL, so each lane runs E / R whole butterflies per stage. Lengths 3 * 2^p use the
// radix-6 and radix-12 butterflies: one exchange fewer than radix 3 followed by radices 2 to 4.
template <int N> struct Radices;
template <> struct Radices<64> { static constexpr int lpl = 16, n = 3; static constexpr int r[3] = {4, 4, 4}; };
template <> struct Radices<96> { static constexpr int lpl = 8, n = 3; static constexpr int r[3] = {6, 4, 4}; };
template <> struct Radices<128> { static constexpr int lpl = 32, n = 4; static constexpr int r[4] = {4, 4, 4, 2}; };
template <> struct Radices<192> { static constexpr int lpl = 16, n = 3; static constexpr int r[3] = {4, 12, 4}; };
template <> struct Radices<256> { static constexpr int lpl = 32, n = 3; static constexpr int r[3] = {8, 8, 4}; };
template <> struct Radices<384> { static constexpr int lpl = 16, n = 3; static constexpr int r[3] = {8, 8, 6}; };
template <> struct Radices<512> { static constexpr int lpl = 32, n = 3; static constexpr int r[3] = {8, 8, 8}; };
template <> struct Radices<768> { static constexpr int lpl = 32, n = 3; static constexpr int r[3] = {8, 8, 12}; };
template <> struct Radices<1024> { static constexpr int lpl = 32, n = 4; static constexpr int r[4] = {8, 8, 8, 2}; };

// Offset of stage S's twiddles in the stage-ordered table of length N: stage s (sub-transforms of
// length NS_s = r_0 ... r_{s-1}, radix R_s) stores exp(2 pi i r k / (NS_s R_s)) at
// k (R_s - 1) + r - 1 for k < NS_s, 0 < r < R_s; the first stage (NS = 1) needs none. Lanes of a
// stage read consecutive k, so the table is read without bank conflicts.
template <int N>
__host__ __device__ constexpr int stage_off(int S) {
  int off = 0, ns = 1;
  for (int s = 0; s < S; ++s) {
    if (ns > 1) off += ns * (Radices<N>::r[s] - 1);
    ns *= Radices<N>::r[s];
  }
  return off;
}

// w^2 .. w^(R-1) from w by squarings and one multiplication per odd power (at most about
// 2 log2 R products deep): p[r - 1] = w^r.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w, float2* p) {
  p[0] = w;
#pragma unroll
  for (int r = 2; r < R; ++r) p[r - 1] = (r % 2 == 0) ? c_mul(p[r / 2 - 1], p[r / 2 - 1]) : c_mul(p[r - 2], w);
}

// One Stockham stage of radix R after sub-transforms of length NS; v[b R + r] is input r of
// butterfly j = lane + b LPL; stw is the stage-ordered twiddle table. POW: read only the first
// twiddle of each butterfly, exp(2 pi i k / (NS R)), and form the others as its powers (less
// shared-memory traffic, more arithmetic: the X/Y passes, which are bound by the former);
// otherwise read all R - 1 (the Z pass, whose arithmetic is the tighter limit).
template <int N, int LPL, int R, int NS, int OFF, bool POW>
__device__ __forceinline__ void stage_compute(float2* v, int lane, const float2* stw) {
  constexpr int BPL = N / (R * LPL);
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int j = lane + b * LPL;
    const int k = j % NS;
    if (NS > 1) {
      if constexpr (POW) {
        float2 w[R - 1];
        twiddle_powers<R>(stw[OFF + k * (R - 1)], w);
#pragma unroll
        for (int r = 1; r < R; ++r) v[b * R + r] = c_mul(v[b * R + r], w[r - 1]);
      } else {
#pragma unroll
        for (int r = 1; r < R; ++r) v[b * R + r] = c_mul(v[b * R + r], stw[OFF + k * (R - 1) + (r - 1)]);
      }
    }
    Dft<float2, R>::run(v + b * R);
  }
}

template <int N, int LPL, int R, int NS>
__device__ __forceinline__ void stage_store(float2* buf, const float2* v, int lane) {
  constexpr int BPL = N / (R * LPL);
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int j = lane + b * LPL;
    const int k = j % NS;
    const int d = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[padn<N>(d + r * NS)] = v[b * R + r];
  }
}

template <int N, int LPL, int R>
__device__ __forceinline__ void stage_load(const float2* buf, float2* v, int lane) {
  constexpr int BPL = N / (R * LPL);
#pragma unroll
  for (int b = 0; b < BPL; ++b) {
    const int j = lane + b * LPL;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = buf[padn<N>(j + r * (N / R))];
  }
}

// Inverse FFT of one line held by LPL lanes: on entry v[b R1 + r] = x[lane + b LPL + r N/R1],
// on exit v[b RL + r] = y[lane + b LPL + r N/RL] (R1, RL the first and last radices).
template <int N, int LPL, int S, int NS, bool POW = true>
__device__ __forceinline__ void warp_fft_from(float2* v, float2* buf, int lane, const float2* stw) {
  constexpr int R = Radices<N>::r[S];
  stage_compute<N, LPL, R, NS, stage_off<N>(S), POW>(v, lane, stw);
  if constexpr (S + 1 < Radices<N>::n) {
    constexpr int R2 = Radices<N>::r[S + 1];
    __syncwarp();
    stage_store<N, LPL, R, NS>(buf, v, lane);
    __syncwarp();
    stage_load<N, LPL, R2>(buf, v, lane);
    warp_fft_from<N, LPL, S + 1, NS * R, POW>(v, buf, lane, stw);
  }
}

template <int N> __host__ __device__ constexpr int first_radix() { return Radices<N>::r[0]; }
template <int N> __host__ __device__ constexpr int last_radix() { return Radices<N>::r[Radices<N>::n - 1]; }

// ---------------------------------------------------------------- X and Y passes
// XPASS: lines along x at (shell n, k_y = it.u, k_z = it.v0 ..), input the half spectrum of the
//        Ng grid (shell mask and optional Kaiser factor applied on load), output G1[x][k_y][k_z].
// else : lines along y at (shell n, x = it.u, k_z = it.v0 ..), input G1, output G2[x][y][k_z].
// N is the side of the evaluation grid (the transform length); kLines lines per block.
template <int N> struct XY {
  static constexpr int kLpl = Radices<N>::lpl;
  static constexpr int kThreads = kLines * kLpl;
};

// Persistent blocks: block b takes items b, b + gridDim.x, ... The input tile of the next item is
// fetched with cp.async (zero-filled outside the shell) into the second of two tile buffers while
// the current item is transformed, so its global-load latency is hidden; the X pass applies the
// Kaiser factor when it reads the tile (counting fields, which have no spectrum, are stored
// directly). The line buffers of the transform overlay the current item's tile once every line
// has read it, so a block holds two regions of max(tile, line buffers) and four blocks fit an SM
// at length 384.
template <int N> __host__ __device__ constexpr int xy_region(int rmax) {
  return 2 * rmax * kTileLd > kLines * line_ld<N>() ? 2 * rmax * kTileLd : kLines * line_ld<N>();
}
// Register budget: as many blocks per SM as the shared memory admits at the longest lines of
// each length (4 up to 384 points, 3 at 512, 2 beyond), so long lines keep their points in
// registers instead of spilling for blocks that could not be resident anyway.
template <int N> __host__ __device__ constexpr int xy_min_blocks() { return N <= 384 ? 4 : N <= 512 ? 3 : 2; }
template <int N, bool XPASS>
__global__ void __launch_bounds__(XY<N>::kThreads, xy_min_blocks<N>()) xy_warp_kernel(PassArgs a, int n_items) {
  constexpr int LPL = XY<N>::kLpl;
  constexpr int NT = XY<N>::kThreads;
  constexpr int E = N / LPL;
  constexpr int kBufLd = line_ld<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);  // N entries exp(2 pi i t / N)
  const int region = xy_region<N>(a.rmax);  // two regions: a tile, or once it is read, the line buffers
  float2* tiles = tw + N;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NT) tw[i] = static_cast<const float2*>(a.stw)[i];
  // ---- input tile [row = k + r - 1][line] of an item: issue the copies (one commit group)
  auto issue = [&](int item, float2* tile) {
    const Item it = a.items[item];
    const ShellGeom g = a.geom[it.n];
    const int r = g.r;
    const int w = 2 * r - 1;
    if (XPASS) {
      const float2* spec = static_cast<const float2*>(a.spec);
      const int ng = a.ng;  // side of the input spectrum's grid
      const int ky = it.u;
      const int iy = ky < 0 ? ky + ng : ky;
      const int hz = ng / 2 + 1;
      for (int idx = tid; idx < w * kLines; idx += NT) {
        const int l = idx & (kLines - 1);
        const int row = idx >> 3;
        const int mx = row - (r - 1);
        const int kz = it.v0 + l;
        const int q = mx * mx + ky * ky + kz * kz;
        const bool in = l < it.cnt && q >= g.qlo && q < g.qhi;
        if (spec) {
          const int ix = mx < 0 ? mx + ng : mx;
          const float2* src = in ? spec + ((long long)ix * ng + iy) * hz + kz : spec;
          ptx::cp_async8_zfill(tile + row * kTileLd + l, src, in ? 8u : 0u);
        } else {
          tile[row * kTileLd + l] = in ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
        }
      }
    } else {
      const float2* g1 = static_cast<const float2*>(a.g1) + g.g1_off;
      const int x = it.u;
      for (int idx = tid; idx < w * kLines; idx += NT) {
        const int l = idx & (kLines - 1);
        const int row = idx >> 3;
        const int ky = row - (r - 1);
        const int kz = it.v0 + l;
        const bool in = l < it.cnt && ky * ky + kz * kz < g.qhi;
        const float2* src = in ? g1 + ((long long)x * w + row) * r + kz : g1;
        ptx::cp_async8_zfill(tile + row * kTileLd + l, src, in ? 8u : 0u);
      }
    }
    ptx::cp_async_commit();
  };
  int k = 0;
  if (blockIdx.x < n_items) issue(blockIdx.x, tiles);
  const int stride = (int)gridDim.x;
  for (int item = blockIdx.x; item < n_items; item += stride, ++k) {
    float2* tile = tiles + (size_t)(k & 1) * region;
    float2* bufs = tile;
    const int next = item + stride;
    if (next < n_items) {
      // the next tile goes where the previous item's line buffers were read out
      if (k > 0) __syncthreads();
      issue(next, tiles + (size_t)((k + 1) & 1) * region);
      ptx::cp_async_wait<1>();  // this item's copies (issued one iteration earlier) have landed
    } else {
      ptx::cp_async_wait<0>();
    }
    const Item it = a.items[item];
    const ShellGeom g = a.geom[it.n];
    const int r = g.r;
    const int w = 2 * r - 1;
    __syncthreads();  // the tile is complete; the previous item's read-out of bufs is done
    // ---- one line per LPL lanes
    {
      constexpr int R1 = first_radix<N>();
      constexpr int BPL = N / (R1 * LPL);
      const int l = tid / LPL;
      const int lane = tid & (LPL - 1);
      float2 v[E];
#pragma unroll
      for (int b = 0; b < BPL; ++b)
#pragma unroll
        for (int rr = 0; rr < R1; ++rr) {
          const int pos = lane + b * LPL + rr * (N / R1);
          const int kk = pos < N / 2 ? pos : pos - N;
          const int row = kk + r - 1;
          float2 t = (row >= 0 && row < w) ? tile[row * kTileLd + l] : make_float2(0.f, 0.f);
          if (XPASS && a.rsd) {  // Kaiser factor (Eq. (3.4)) of the shell's modes, in FP32
            const int kz = it.v0 + l;
            const int q = kk * kk + it.u * it.u + kz * kz;
            if (row >= 0 && row < w && l < it.cnt && q >= g.qlo && q < g.qhi) {
              const float fac = 1.0f + (float)a.beta * ((float)(kz * kz) / (float)q);
              t.x *= fac;
              t.y *= fac;
            }
          }
          v[b * R1 + rr] = t;
        }
      __syncthreads();  // every line has read the tile its buffers overlay
      float2* buf = bufs + (size_t)l * kBufLd;
      warp_fft_from<N, LPL, 0, 1>(v, buf, lane, tw);
      constexpr int RL = last_radix<N>();
      constexpr int BPLL = N / (RL * LPL);
      __syncwarp();
#pragma unroll
      for (int b = 0; b < BPLL; ++b)
#pragma unroll
        for (int rr = 0; rr < RL; ++rr) buf[padn<N>(lane + b * LPL + rr * (N / RL))] = v[b * RL + rr];
    }
    __syncthreads();
    // ---- output tile -> global, contiguous along k_z
    float2* out;
    long long row_stride;
    if (XPASS) {
      out = static_cast<float2*>(a.g1) + g.g1_off + (long long)(it.u + r - 1) * r + it.v0;
      row_stride = (long long)w * r;
    } else {
      out = static_cast<float2*>(a.g2) + g.g2_off + (long long)it.u * N * r + it.v0;
      row_stride = r;
    }
    for (int idx = tid; idx < N * kLines; idx += NT) {
      const int l = idx & (kLines - 1);
      const int y = idx >> 3;
      if (l < it.cnt) out[y * row_stride + l] = bufs[(size_t)l * kBufLd + padn<N>(y)];
    }
  }
}

// ---------------------------------------------------------------- Z pass
// SLAB: only the x-slab of a.slab_x0 / a.slab_nx, fields [n][x - slab_x0][y][z] (FP32, or split
// planes when a.split_lo != 0).
// Register budget: 4 blocks per SM (64 registers) unless the line is long (768, 1024: 24-32
// points per lane spill below 128 registers).
template <int S>
__host__ __device__ constexpr int z_min_blocks() { return S >= 768 ? 2 : 4; }

template <int S, bool SLAB>
__global__ void __launch_bounds__(kZThreads, z_min_blocks<S>()) z_warp_kernel(PassArgs a, long long n_lines) {
  constexpr int M = S / 2;
  constexpr int LPL = Radices<M>::lpl;
  constexpr int LPW = 32 / LPL;  // lines per warp at a time
  constexpr int E = M / LPL;
  constexpr int kBufLd = pad_len<M>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);  // M entries: stage twiddles of length M
  float2* wk = tw + M;                               // M entries: exp(2 pi i k / S), k < M
  float2* bufs = wk + M;
  uint32_t* zmask = reinterpret_cast<uint32_t*>(bufs + (size_t)(kZThreads / 32) * LPW * kBufLd);  // S entries
  const int tid = threadIdx.x;
  for (int i = tid; i < M; i += kZThreads) {
    tw[i] = static_cast<const float2*>(a.stw_half)[i];
    wk[i] = static_cast<const float2*>(a.tw)[i];
  }
  if (a.n_zlev > 0)
    for (int i = tid; i < S; i += kZThreads) zmask[i] = a.zmask[i];
  __syncthreads();
  const int warp = tid >> 5;
  const int sub = (tid & 31) / LPL;  // line slot inside the warp
  const int lane = tid & (LPL - 1);
  float2* buf = bufs + (size_t)(warp * LPW + sub) * kBufLd;
  const long long plane = (long long)S * S;
  const long long stride = (long long)gridDim.x * (kZThreads / 32) * LPW;
  constexpr int R1 = first_radix<M>();
  constexpr int BPL = M / (R1 * LPL);
  constexpr int RL = last_radix<M>();
  constexpr int BPLL = M / (RL * LPL);
  for (long long line = ((long long)blockIdx.x * (kZThreads / 32) + warp) * LPW + sub; line < n_lines;
       line += stride) {
    const long long per = SLAB ? (long long)a.slab_nx * S : plane;  // lines of one shell
    const int n = (int)(line / per);
    const long long xyl = line - (long long)n * per;                  // line within the shell's output
    const long long xy = SLAB ? (long long)a.slab_x0 * S + xyl : xyl;  // (x, y) on the grid
    const ShellGeom g = a.geom[n];
    const int r = g.r;
    const float2* src = static_cast<const float2*>(a.g2) + g.g2_off + xy * r;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < BPL; ++b)
#pragma unroll
      for (int rr = 0; rr < R1; ++rr) {
        const int k = lane + b * LPL + rr * (M / R1);
        const float2 xk = k < r ? src[k] : make_float2(0.f, 0.f);
        const float2 xm = (k > 0 && M - k < r) ? src[M - k] : make_float2(0.f, 0.f);
        const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);                // X[k] + conj X[M-k]
        const float2 o = c_mul(make_float2(xk.x - xm.x, xk.y + xm.y), wk[k]);  // (X[k] - conj X[M-k]) W^k
        v[b * R1 + rr] = make_float2(e.x - o.y, e.y + o.x);                    // e + i o
      }
    warp_fft_from<M, LPL, 0, 1, false>(v, buf, lane, tw);
    const long long off = (long long)n * S * per + xyl * S;  // first voxel of the line
    if (a.split_lo == 0) {
      float2* dst = reinterpret_cast<float2*>(static_cast<float*>(a.fields) + off);
#pragma unroll
      for (int b = 0; b < BPLL; ++b)
#pragma unroll
        for (int rr = 0; rr < RL; ++rr) dst[lane + b * LPL + rr * (M / RL)] = v[b * RL + rr];
    } else {
      // split fields: bf16 high parts of the voxel pair (2k, 2k + 1) in one word, low parts in
      // the word split_lo further
      uint32_t* hi = static_cast<uint32_t*>(a.fields) + off / 2;
#pragma unroll
      for (int b = 0; b < BPLL; ++b)
#pragma unroll
        for (int rr = 0; rr < RL; ++rr) {
          const float2 x = v[b * RL + rr];
          uint32_t h, l;
          ptx::split_bf16x2(ptx::f2_pack(x.x, x.y), h, l);
          const int k = lane + b * LPL + rr * (M / RL);
          hi[k] = h;
          hi[a.split_lo + k] = l;
        }
      // coarser levels: lines with x and y multiples of the level's stride, every t-th voxel
      // (plans streaming x-slabs have one level)
      if (!SLAB && a.n_zlev > 0) {
        const int x = (int)(xy / S);
        const int y = (int)(xy - (long long)x * S);
        uint32_t mask = zmask[x] & zmask[y];
        while (mask != 0) {
          const int l = __ffs(mask) - 1;
          mask &= mask - 1;
          const ZLevel L = a.zlev[l];
          const int j = L.loc[n];
          if (j < 0) continue;
          uint16_t* lh = L.dst + (((long long)j * L.g + __float2int_rn(x * L.rt)) * L.g + __float2int_rn(y * L.rt)) * L.g;
          // power-of-two strides t with t / 2 dividing every element offset b LPL + rr M / RL: a lane
          // keeps all its even z (z = 2k, k = lane + offset) or none, at z / t = k / (t / 2)
          constexpr int kG = (LPL % (M / RL) == 0) ? (M / RL) : ((M / RL) % LPL == 0 ? LPL : 1);
          const int ht = L.t >> 1;
          if ((L.t & (L.t - 1)) == 0 && kG % ht == 0) {
            if (lane % ht == 0) {
              const int sh = __ffs(ht) - 1;
#pragma unroll
              for (int b = 0; b < BPLL; ++b)
#pragma unroll
                for (int rr = 0; rr < RL; ++rr) {
                  const int zz = (lane + b * LPL + rr * (M / RL)) >> sh;
                  const float2 x2 = v[b * RL + rr];
                  uint32_t h, lo;
                  ptx::split_bf16x2(ptx::f2_pack(x2.x, x2.y), h, lo);
                  lh[zz] = (uint16_t)(h & 0xFFFFu);
                  lh[L.lo_off + zz] = (uint16_t)(lo & 0xFFFFu);
                }
            }
            continue;
          }
#pragma unroll
          for (int b = 0; b < BPLL; ++b)
#pragma unroll
            for (int rr = 0; rr < RL; ++rr) {
              const int k = lane + b * LPL + rr * (M / RL);
              // z = 2k and 2k + 1 on the level's grid: z / t by the rounded reciprocal, kept when exact
              const int q0 = __float2int_rn((2 * k) * L.rt), q1 = __float2int_rn((2 * k + 1) * L.rt);
              const bool e0 = q0 * L.t == 2 * k, e1 = q1 * L.t == 2 * k + 1;
              if (e0 || e1) {
                const float2 x2 = v[b * RL + rr];
                uint32_t h, lo;
                ptx::split_bf16x2(ptx::f2_pack(x2.x, x2.y), h, lo);
                if (e0) {
                  lh[q0] = (uint16_t)(h & 0xFFFFu);
                  lh[L.lo_off + q0] = (uint16_t)(lo & 0xFFFFu);
                }
                if (e1) {
                  lh[q1] = (uint16_t)(h >> 16);
                  lh[L.lo_off + q1] = (uint16_t)(lo >> 16);
                }
              }
            }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- forward (adjoint) passes
// The transposes of the passes above, for the gradient: a real field G_n on the S grid is taken
// to sum_x G_n(x) e^{+i k.x} on the modes of shell n only, by the same unnormalised e^{+i}
// transforms applied in the opposite order with pruned outputs:
//   ZF: lines (n, x, y) along z, real input, keep k_z < r      -> H1[x][y][k_z]   (G2 layout)
//   YF: lines (n, x, k_z) along y, keep |k_y| < r              -> H2[x][k_y][k_z] (G1 layout)
//   XF: lines (n, k_y, k_z) along x, keep the shell's modes    -> conj(.) K(k) scale into the
//       half spectrum of the ng grid (Eq. (3.4) factor K when the plan has RSD).
// With a.slab_nx > 0 the ZF pass takes the lines of one x-slab, G_n laid out [n][x - slab_x0][y][z].
template <int S>
__global__ void __launch_bounds__(kZThreads) zf_warp_kernel(PassArgs a, const float* gfield, long long n_lines) {
  constexpr int LPL = Radices<S>::lpl;
  constexpr int LPW = 32 / LPL;
  constexpr int E = S / LPL;
  constexpr int kBufLd = pad_len<S>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);  // stage twiddles of length S
  float2* bufs = tw + S;
  const int tid = threadIdx.x;
  for (int i = tid; i < S; i += kZThreads) tw[i] = static_cast<const float2*>(a.stw)[i];
  __syncthreads();
  const int warp = tid >> 5;
  const int sub = (tid & 31) / LPL;
  const int lane = tid & (LPL - 1);
  float2* buf = bufs + (size_t)(warp * LPW + sub) * kBufLd;
  const long long plane = (long long)S * S;
  const long long stride = (long long)gridDim.x * (kZThreads / 32) * LPW;
  constexpr int R1 = first_radix<S>();
  constexpr int BPL = S / (R1 * LPL);
  constexpr int RL = last_radix<S>();
  constexpr int BPLL = S / (RL * LPL);
  for (long long line = ((long long)blockIdx.x * (kZThreads / 32) + warp) * LPW + sub; line < n_lines;
       line += stride) {
    const long long per = a.slab_nx ? (long long)a.slab_nx * S : plane;  // lines of one shell
    const int n = (int)(line / per);
    const long long xyl = line - (long long)n * per;
    const long long xy = (long long)a.slab_x0 * S + xyl;  // slab_x0 is 0 without slabs
    const ShellGeom g = a.geom[n];
    const int r = g.r;
    const float* src = gfield + (long long)n * S * per + xyl * S;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < BPL; ++b)
#pragma unroll
      for (int rr = 0; rr < R1; ++rr) v[b * R1 + rr] = make_float2(src[lane + b * LPL + rr * (S / R1)], 0.f);
    warp_fft_from<S, LPL, 0, 1>(v, buf, lane, tw);
    float2* dst = static_cast<float2*>(a.g2) + g.g2_off + xy * r;
#pragma unroll
    for (int b = 0; b < BPLL; ++b)
#pragma unroll
      for (int rr = 0; rr < RL; ++rr) {
        const int k = lane + b * LPL + rr * (S / RL);
        if (k < r) dst[k] = v[b * RL + rr];
      }
  }
}

// XPASS = false: YF (input H1 = G2 layout, output H2 = G1 layout).
// XPASS = true : XF (input H2, output the ng half spectrum `a.fields` reinterpreted as complex).
template <int N, bool XPASS>
__global__ void __launch_bounds__(XY<N>::kThreads) xyf_warp_kernel(PassArgs a, float scale) {
  constexpr int LPL = XY<N>::kLpl;
  constexpr int NT = XY<N>::kThreads;
  constexpr int E = N / LPL;
  constexpr int kBufLd = line_ld<N>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);  // N
  float2* bufs = tw + N;                               // kLines x kBufLd
  float2* tile = bufs + (size_t)kLines * kBufLd;       // N x kTileLd input, then (2r-1) x kTileLd output
  const Item it = a.items[blockIdx.x];
  const ShellGeom g = a.geom[it.n];
  const int r = g.r;
  const int w = 2 * r - 1;
  const int tid = threadIdx.x;
  for (int i = tid; i < N; i += NT) tw[i] = static_cast<const float2*>(a.stw)[i];
  // ---- input tile [position along the line][line], contiguous along k_z in memory
  const float2* src;
  long long row_stride;
  if (XPASS) {
    src = static_cast<const float2*>(a.g1) + g.g1_off + (long long)(it.u + r - 1) * r + it.v0;
    row_stride = (long long)w * r;
  } else {
    src = static_cast<const float2*>(a.g2) + g.g2_off + (long long)it.u * N * r + it.v0;
    row_stride = r;
  }
  for (int idx = tid; idx < N * kLines; idx += NT) {
    const int l = idx & (kLines - 1);
    const int y = idx >> 3;
    tile[y * kTileLd + l] = l < it.cnt ? src[y * row_stride + l] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  {
    constexpr int R1 = first_radix<N>();
    constexpr int BPL = N / (R1 * LPL);
    const int l = tid / LPL;
    const int lane = tid & (LPL - 1);
    float2 v[E];
#pragma unroll
    for (int b = 0; b < BPL; ++b)
#pragma unroll
      for (int rr = 0; rr < R1; ++rr) v[b * R1 + rr] = tile[(lane + b * LPL + rr * (N / R1)) * kTileLd + l];
    float2* buf = bufs + (size_t)l * kBufLd;
    warp_fft_from<N, LPL, 0, 1>(v, buf, lane, tw);
    constexpr int RL = last_radix<N>();
    constexpr int BPLL = N / (RL * LPL);
    __syncwarp();
#pragma unroll
    for (int b = 0; b < BPLL; ++b)
#pragma unroll
      for (int rr = 0; rr < RL; ++rr) buf[padn<N>(lane + b * LPL + rr * (N / RL))] = v[b * RL + rr];
  }
  __syncthreads();
  // ---- keep the positions |k| <= r - 1: row = k + r - 1
  if (XPASS) {
    float2* spec = reinterpret_cast<float2*>(a.fields);
    const int ng = a.ng;
    const int hz = ng / 2 + 1;
    const int ky = it.u;
    const int iy = ky < 0 ? ky + ng : ky;
    for (int idx = tid; idx < w * kLines; idx += NT) {
      const int l = idx & (kLines - 1);
      const int row = idx >> 3;
      const int kx = row - (r - 1);
      const int kz = it.v0 + l;
      const int q = kx * kx + ky * ky + kz * kz;
      if (l < it.cnt && q >= g.qlo && q < g.qhi) {
        float2 val = bufs[(size_t)l * kBufLd + padn<N>(kx < 0 ? kx + N : kx)];
        float fac = scale;
        if (a.rsd) fac *= (float)(1.0 + a.beta * (double)(kz * kz) / (double)q);
        const int ix = kx < 0 ? kx + ng : kx;
        spec[((long long)ix * ng + iy) * hz + kz] = make_float2(val.x * fac, -val.y * fac);
      }
    }
  } else {
    float2* dst = static_cast<float2*>(a.g1) + g.g1_off + (long long)it.u * w * r + it.v0;
    for (int idx = tid; idx < w * kLines; idx += NT) {
      const int l = idx & (kLines - 1);
      const int row = idx >> 3;
      const int ky = row - (r - 1);
      if (l < it.cnt) dst[(long long)row * r + l] = bufs[(size_t)l * kBufLd + padn<N>(ky < 0 ? ky + N : ky)];
    }
  }
}

template <int N, bool XPASS>
bsp_status launch_xyf(const PassArgs& a, int n_items, float scale, cudaStream_t s) {
  if (n_items == 0) return BSP_OK;
  const size_t smem = ((size_t)N + (size_t)kLines * line_ld<N>() + (size_t)N * kTileLd) * sizeof(float2);
  BSP_CUDA(cudaFuncSetAttribute(xyf_warp_kernel<N, XPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  xyf_warp_kernel<N, XPASS><<<n_items, XY<N>::kThreads, smem, s>>>(a, scale);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template <int S>
bsp_status launch_zf(const PassArgs& a, const float* gfield, long long n_lines, int n_sm, cudaStream_t s) {
  constexpr int LPW = 32 / Radices<S>::lpl;
  const size_t smem = ((size_t)S + (size_t)(kZThreads / 32) * LPW * pad_len<S>()) * sizeof(float2);
  BSP_CUDA(cudaFuncSetAttribute(zf_warp_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, zf_warp_kernel<S>, kZThreads, smem));
  long long blocks = (long long)std::max(per_sm, 1) * n_sm;
  const long long need = (n_lines + (kZThreads / 32) * LPW - 1) / ((kZThreads / 32) * LPW);
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  zf_warp_kernel<S><<<(unsigned)blocks, kZThreads, smem, s>>>(a, gfield, n_lines);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template <int N, bool XPASS>
bsp_status launch_xy(const PassArgs& a, int n_items, int n_sm, cudaStream_t s) {
  if (n_items == 0) return BSP_OK;
  // two regions, each holding a tile of 2 r - 1 rows of the largest shell or, once it is read,
  // the line buffers
  const size_t smem = ((size_t)N + 2 * (size_t)xy_region<N>(a.rmax)) * sizeof(float2);
  BSP_CUDA(cudaFuncSetAttribute(xy_warp_kernel<N, XPASS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xy_warp_kernel<N, XPASS>, XY<N>::kThreads, smem));
  long long blocks = std::min<long long>((long long)std::max(per_sm, 1) * std::max(n_sm, 1), n_items);
  if (!XPASS && a.grid_blocks > 0) blocks = std::min<long long>(a.grid_blocks, n_items);
  xy_warp_kernel<N, XPASS><<<(unsigned)blocks, XY<N>::kThreads, smem, s>>>(a, n_items);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

template <int S>
bsp_status launch_z(const PassArgs& a, long long n_lines, int n_sm, cudaStream_t s) {
  constexpr int M = S / 2;
  constexpr int LPW = 32 / Radices<M>::lpl;
  const size_t smem = ((size_t)2 * M + (size_t)(kZThreads / 32) * LPW * pad_len<M>()) * sizeof(float2) +
                      (a.n_zlev > 0 ? (size_t)S * sizeof(uint32_t) : 0);
  auto kern = a.slab_nx > 0 ? z_warp_kernel<S, true> : z_warp_kernel<S, false>;
  BSP_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BSP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kZThreads, smem));
  long long blocks = (long long)std::max(per_sm, 1) * n_sm;
  const long long need = (n_lines + (kZThreads / 32) * LPW - 1) / ((kZThreads / 32) * LPW);
  if (a.grid_blocks > 0) blocks = a.grid_blocks;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  kern<<<(unsigned)blocks, kZThreads, smem, s>>>(a, n_lines);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}

}  // namespace

template <int N>
static void stage_table(std::vector<float2>& out) {
  out.clear();
  int ns = 1;
  for (int s = 0; s < Radices<N>::n; ++s) {
    const int R = Radices<N>::r[s];
    if (ns > 1)
      for (int k = 0; k < ns; ++k)
        for (int r = 1; r < R; ++r) {
          const double ang = 2.0 * 3.14159265358979323846 * (double)r * (double)k / (double)(ns * R);
          out.push_back(make_float2((float)cos(ang), (float)sin(ang)));
        }
    ns *= R;
  }
  out.resize(N, make_float2(0.f, 0.f));
}

bool warp_stage_table(int n, std::vector<float2>& out) {
  switch (n) {
#define X(N) case N: stage_table<N>(out); return true;
    X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)
#undef X
  }
  return false;
}

bool warp_fft_supported(int s) {
  return s == 128 || s == 192 || s == 256 || s == 384 || s == 512 || s == 768 || s == 1024;
}
int warp_fft_lines() { return kLines; }

#define BSP_WARP_SIZES(X) X(128) X(192) X(256) X(384) X(512) X(768) X(1024)

bsp_status launch_warp_xpass(const PassArgs& a, int n_items, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_xy<S, true>(a, n_items, a.n_sm, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

bsp_status launch_warp_ypass(const PassArgs& a, int n_items, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_xy<S, false>(a, n_items, a.n_sm, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

bsp_status launch_warp_zpass(const PassArgs& a, long long n_lines, int n_sm, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_z<S>(a, n_lines, n_sm, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

bsp_status launch_warp_zfpass(const PassArgs& a, const float* gfield, long long n_lines, int n_sm, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_zf<S>(a, gfield, n_lines, n_sm, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

bsp_status launch_warp_yfpass(const PassArgs& a, int n_items, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_xyf<S, false>(a, n_items, 1.f, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

bsp_status launch_warp_xfpass(const PassArgs& a, int n_items, float scale, cudaStream_t s) {
  switch (a.ngs) {
#define X(S) case S: return launch_xyf<S, true>(a, n_items, scale, s);
    BSP_WARP_SIZES(X)
#undef X
  }
  return fail_c(BSP_ERR_NOT_SUPPORTED, "warp FFT: unsupported grid");
}

}  // namespace bsp
