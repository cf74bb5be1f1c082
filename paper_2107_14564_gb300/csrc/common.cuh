// Shared device helpers and the internal plan layout of the bispectrum library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "bispec.h"

namespace bsp {

// ---------------------------------------------------------------- complex arithmetic
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx = typename Cplx<T>::type;

template <typename C> __device__ __forceinline__ C c_make(decltype(C::x) re, decltype(C::x) im) {
  C r; r.x = re; r.y = im; return r;
}
template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return c_make<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return c_make<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
  return c_make<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C c_conj(C a) { return c_make<C>(a.x, -a.y); }
// multiply by +i
template <typename C> __device__ __forceinline__ C c_muli(C a) { return c_make<C>(-a.y, a.x); }
template <typename C> __device__ __forceinline__ C c_scale(C a, decltype(C::x) s) { return c_make<C>(a.x * s, a.y * s); }

// ---------------------------------------------------------------- FFT stage list
constexpr int kMaxStages = 12;
struct FftStages {
  int n;                  // transform length
  int nst;                // number of stages
  int radix[kMaxStages];  // radices, product = n
};

// Threads per FFT block and complex elements held per thread in one stage.
constexpr int kFftThreads = 256;
template <typename T> struct FftElems;
template <> struct FftElems<float> { static constexpr int value = 32; };
template <> struct FftElems<double> { static constexpr int value = 16; };

// ---------------------------------------------------------------- work items of the passes
// X pass: lines along x at fixed (shell n, ky, kz0..kz0+cnt)
// Y pass: lines along y at fixed (shell n, x, kz0..kz0+cnt)
// Z pass: lines along z at fixed (shell n, x, y0..y0+cnt)
struct Item { int n, u, v0, cnt; };

struct ShellGeom {
  int qlo, qhi;        // modes with qlo <= |m|^2 < qhi
  int r;               // |m_i| <= r - 1 for every mode of the shell
  int pad;
  long long g1_off;    // complex offset of this shell in the X-pass buffer [x][2r-1][r]
  long long g2_off;    // complex offset in the Y-pass buffer [x][y][r]
};

struct PassArgs {
  const void* spec;       // half spectrum (complex T), or null for the unit counting input
  void* g1;               // X-pass output
  void* g2;               // Y-pass output
  void* fields;           // Z-pass output, [n][x][y][z] real T
  const void* tw;         // twiddles exp(+2 pi i j / ngs), j < ngs (complex T)
  const void* stw;        // warp kernels: stage-ordered twiddles of length ngs (float2)
  const void* stw_half;   // warp kernels: stage-ordered twiddles of length ngs / 2
  const ShellGeom* geom;  // per shell
  const Item* items;      // work items of this pass
  int ng;                 // side of the input spectrum's grid
  int ngs;                // side of the evaluation grid (transform length), <= ng
  int rsd;
  double beta;
  int kweight;            // generic X pass, counting input only: mode value |k| / k_f instead of 1
  int grid_blocks;        // warp Y and Z passes: blocks of the persistent grid (0: as many as fit)
  int slab_x0, slab_nx;   // Z passes: only x in [slab_x0, slab_x0 + slab_nx) of the evaluation grid,
                          // fields laid out [n][x - slab_x0][y][z]; slab_nx = 0: the whole grid
  FftStages st;           // stage list of this pass's line length
  int rmax;               // largest r of all shells
  int n_sm;               // SMs of the device (grid size of the persistent warp kernels)
  long long split_lo;     // warp Z pass: 0 writes FP32 fields; otherwise bf16 high parts [n][x][y][z]
                          // at `fields` and low parts split_lo 32-bit words further (split fields)
  // split warp Z pass: also write the split fields of the coarser contraction levels
  const struct ZLevel* zlev;  // n_zlev levels
  const uint32_t* zmask;      // [ngs]: bit l set when coordinate i is a multiple of level l's stride
  int n_zlev;
};

// A coarser contraction level the split Z pass samples: voxel (x, y, z) of the evaluation grid with
// all three coordinates multiples of the stride t goes to (x / t, y / t, z / t) of the level.
struct ZLevel {
  uint16_t* dst;      // [2][nsh][g^3] split planes
  long long lo_off;   // nsh * g^3: offset of the low plane (elements)
  const int* loc;     // [ns]: the level's field index of each shell, -1 if unused
  int g;              // level side
  int t;              // stride: evaluation-grid side / g
  float rt;           // 1 / t (x / t = rint(x rt) for the multiples x of t below 2^24)
};

// Warp-per-line FP32 passes (bispec_fft_warp.cu) for evaluation grids 2^p and 3 * 2^p from
// 128 to 1024; X/Y items hold at most warp_fft_lines() lines.
bool warp_fft_supported(int ngs);
// Stage-ordered twiddle table of a warp FFT length (n entries, zero padded); false if unsupported.
bool warp_stage_table(int n, std::vector<float2>& out);
int warp_fft_lines();
bsp_status launch_warp_xpass(const PassArgs& a, int n_items, cudaStream_t s);
bsp_status launch_warp_ypass(const PassArgs& a, int n_items, cudaStream_t s);
bsp_status launch_warp_zpass(const PassArgs& a, long long n_lines, int n_sm, cudaStream_t s);
// Forward (adjoint) passes: real fields gfield [n][S^3] -> per-shell modes, written as
// conj(sum_x G e^{+ik.x}) * K * scale into the ng half spectrum a.fields (complex64).
bsp_status launch_warp_zfpass(const PassArgs& a, const float* gfield, long long n_lines, int n_sm, cudaStream_t s);
bsp_status launch_warp_yfpass(const PassArgs& a, int n_items, cudaStream_t s);
bsp_status launch_warp_xfpass(const PassArgs& a, int n_items, float scale, cudaStream_t s);

// ---------------------------------------------------------------- contraction tables
// A tile covers up to 4 consecutive pairs and 4 consecutive c shells; map[16] gives the kept
// bin of output (i, j) or -1.
struct Tile { int p0, np, c0, pad; };

// ---------------------------------------------------------------- error handling
void set_error(const std::string& msg);
void set_error_c(const char* msg);  // no allocation
bsp_status fail(bsp_status s, const std::string& msg);
bsp_status fail_c(bsp_status s, const char* msg);  // no allocation
bsp_status cuda_fail(cudaError_t e, const char* what);

#define BSP_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::bsp::cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------- launchers (bispec_fft.cu)
template <typename T>
bsp_status launch_xpass(const PassArgs& a, int n_items, int lines, cudaStream_t s);
template <typename T>
bsp_status launch_ypass(const PassArgs& a, int n_items, int lines, cudaStream_t s);
template <typename T>
bsp_status launch_zpass(const PassArgs& a, int n_items, int lines, cudaStream_t s);
// out[j][v] = f[pairs[j].x][v] * f[pairs[j].y][v] for v < nvox (order-4 plans: the product fields
// d_c d_e through which sum_x d_a d_b d_c d_e becomes a triple sum)
template <typename T>
bsp_status launch_pair_fields(const void* f, long long nvox, const int2* pairs, int np, void* out, int n_sm,
                              cudaStream_t s);
// 2D rings: C2C along x of the (n, k_y) lines -> G[n][x][k_y < r] (the C2R along y is the Z
// pass kernel run on those rows, see plan_passes_2d)
template <typename T>
bsp_status launch_ring_xpass(const PassArgs& a, int n_items, int lines, cudaStream_t s);
template <typename T>
bsp_status launch_twiddles(void* tw, int ng, cudaStream_t s);

// ---------------------------------------------------------------- launchers (bispec_contract.cu)
struct ContractArgs {
  const void* fields;     // [ns][nvox] real T
  long long nvox;
  int ns;
  const Tile* tiles;
  const int2* pairs;      // (a, b)
  const int* tile_map;    // [ntiles][16]
  int ntiles;
  double* partial;        // [gridx][ntiles][16]
  int gridx;
  double* msum;           // [n_out]
  int n_out;
  double scale;           // msum = scale * (sum over the evaluation grid)
  int accumulate;         // reduce: msum += instead of msum = (later x-slabs of one sum)
};
template <typename T>
bsp_status launch_contract_simt(const ContractArgs& a, cudaStream_t s);
bsp_status launch_reduce_partials(const ContractArgs& a, cudaStream_t s);
template <typename T>
bsp_status launch_decimate(const void* src, int S, const int* shells, int nsh, void* dst, int g, int t, int n_sm,
                           cudaStream_t s);

struct FinalizeArgs {
  const double* msum;
  const double* tsum;
  int n_trip;
  const int* cell_ptr;    // CSR over n_cells cells
  const int* cell_idx;
  int n_cells;
  double norm;            // V_c^3 / V
  double* b_trip;
  double* b_grid;         // may be null
};
bsp_status launch_finalize(const FinalizeArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core contraction
constexpr int kTcVoxelChunk = 64;  // voxels per pipeline stage of the tensor-core contraction
constexpr int kTcSlots = 64;       // pair-group slots of one tile group (a 128-lane M tile of hi/lo rows)
// Split fields: d = d_hi + d_lo with d_hi = bf16(d) and d_lo = bf16(d - d_hi), stored as two
// bf16 planes [2][ns][nvox] (high parts first). The contraction reads them through a 3D tensor
// map (voxel, shell, part) with 64 x NP x 1 boxes and the 128-byte swizzle.
//
// Pairs are packed into groups of up to KT pairs built from three fields (f0, f1, f2) of one
// slot: tile 0 holds the pair (f0, s ? f1 : f0), tile 1 (f0, f2), tile 2 (f1, f2), where s is
// bit 0 of the slot's flags; bit 1 marks a slot holding at least one kept pair.
struct TcArgs {
  long long nvox;           // multiple of kTcVoxelChunk
  int np;                   // shells padded for the MMA N dimension (32 or 64)
  int kt;                   // pair tiles per tile group (1..3; 1..2 when np = 64)
  const int4* groups;       // [n_tg * kTcSlots] (f0, f1, f2, flags)
  int n_tg;                 // tile groups
  int gridy;                // voxel blocks
  long long vox_per_block;  // multiple of kTcVoxelChunk
  float2* partial;          // [gridy][n_tg][kt][kTcSlots][np] run sums as FP32 pairs s + c
  int* error;               // set to 1 when a bounded wait gives up
};
int tc_padded_shells(int ns);
// One warp whose bounded wait on an mbarrier nothing arrives at runs out and sets *error.
bsp_status launch_wait_selftest(int* error, cudaStream_t s);
size_t tc_partial_entries(int n_tg, int kt, int gridy, int np);
bsp_status launch_contract_tc(const TcArgs& a, const CUtensorMap* tmap, cudaStream_t s);
// Encode the tensor map of split fields at `base` ([2][rows][nvox] bf16) for NP-row boxes.
bsp_status encode_split_map(CUtensorMap* map, void* base, long long nvox, int rows, int np);
// Split FP32 fields [ns][nvox] into bf16 planes: hi (n words of two values) at dst, lo at dst + n.
bsp_status launch_split_fields(const float* src, uint32_t* dst, long long n_words, int n_sm, cudaStream_t s);
// One kept bin of the tensor-core contraction: msum[t] = scale * sum_y partial[y * stride + off].
struct TcBin {
  const float2* partial;
  long long stride;
  int gridy;
  int off;
  double scale;
};
// Every bin of every level in one launch (one warp per bin, a fixed summation order); with
// `accumulate` the sums are added to msum (the x-slabs of a budgeted plan).
bsp_status launch_reduce_tc_all(const TcBin* bins, int n, double* msum, cudaStream_t s, bool accumulate = false);

// ---------------------------------------------------------------- gradient (bispec_grad.cu)
bsp_status launch_build_w(const double* g, const double* cnorm, const int* ptr, const int* idx, int n_entries,
                          float* W, cudaStream_t s);
bsp_status launch_adjoint_products(const float* fields, long long nvox, int ns, int np, const int2* pairs,
                                   int npairs, const float* W, float* G, int n_sm, cudaStream_t s);

}  // namespace bsp
