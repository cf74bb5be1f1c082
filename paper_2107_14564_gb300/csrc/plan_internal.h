// Internal declarations shared by the plan construction (bispec_plan.cu) and the estimator and
// entry points (bispec_api.cu): the plan object, its device allocations and the host-side steps.
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace bsp {

// ---------------------------------------------------------------- host-side helpers
inline long long isqrt_ll(long long v) {
  if (v < 0) return -1;
  long long r = (long long)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// FFT stage list: radix 8 while possible, then 4, 2 and 3.
inline bool make_stages(int n, FftStages* st) {
  st->n = n;
  st->nst = 0;
  int m = n;
  while (m % 8 == 0 && st->nst < kMaxStages) { st->radix[st->nst++] = 8; m /= 8; }
  while (m % 4 == 0 && st->nst < kMaxStages) { st->radix[st->nst++] = 4; m /= 4; }
  while (m % 2 == 0 && st->nst < kMaxStages) { st->radix[st->nst++] = 2; m /= 2; }
  while (m % 3 == 0 && st->nst < kMaxStages) { st->radix[st->nst++] = 3; m /= 3; }
  return m == 1;
}

// Device allocation owned by a plan.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace bsp

using namespace bsp;

// One level of the contraction: the bins whose triple products hold only wavevectors with
// components below g_l are summed on a g_l^3 grid (a divisor of the evaluation grid, sampled from
// its fields with stride S / g_l), exact for the same reason the evaluation grid is.
struct ContractLevel {
  int g = 0;                  // grid side
  int stride = 1;             // evaluation-grid side / g
  double scale = 1.0;         // (ng / g)^3
  std::vector<int> shells;    // global shell of each local field index
  std::vector<int> bins;      // kept bins (global indices, ascending) summed on this level
  bool top = false;           // uses the plan's fields directly (all shells, global indices)
  void* fields = nullptr;     // [shells][g^3] for lower levels (split planes [2][shells][g^3] for
                              // tensor-core plans)
  int* d_shells = nullptr;    // source field of each destination field of the level sampling
  CUtensorMap tmap{};         // tensor-core plans: the level's split fields (under a memory
                              // budget: those of a full x-slab)
  CUtensorMap tmap_last{};    // under a memory budget: the last (shorter) x-slab's split fields
  // CUDA-core contraction
  Tile* d_tiles = nullptr;
  int2* d_pairs = nullptr;
  int* d_map = nullptr;       // [ntiles][16] global bin index or -1
  int ntiles = 0, gridx = 0;
  double* partial = nullptr;
  // tensor-core contraction
  int np = 0, kt = 0, n_tg = 0, gridy = 0;  // padded shells, pair tiles per tile group, tile groups
  long long vpb = 0;
  int4* d_tc_groups = nullptr;  // [n_tg * kTcSlots] slot fields and flags (see TcArgs)
  std::vector<int> tc_off;    // partial-sum entry of each of the level's bins
  int gridy_cap = 0;          // voxel blocks the partial-sum buffer holds
  int tune_mult = 1;          // voxel blocks per tile group / SM count chosen by the autotuner (1 without it)
  float2* tc_partial = nullptr;
  int dim = 3;                // 2: a level of a 2D plan (g^2 points)
  long long nvox() const { return dim == 2 ? (long long)g * g : (long long)g * g * g; }
};

constexpr int kNumTune = 3;
constexpr int kTuneMults[kNumTune] = {1, 2, 4};

struct bsp_plan {
  // description
  int ng = 0, ns = 0, n_mu = 0, n_t = 0, rsd = 0, prec = 0;
  int autotune = 0;
  int y_blocks = 0, z_blocks = 0;  // warp Y and Z pass grids picked by autotune_passes (0: as many as fit)
  int k1_merge = 1;         // k1 shells per (mu, t) cell group
  int label_k = BSP_LABEL_SHELL_MEAN;
  int dim = 3;              // 2: Ng^2 square with annular rings (Sec. 2.1); 3: Ng^3 cube with shells
  int order = 3;            // 3: bispectrum; 4: binned 4-point sum over (a, b, c, e)
  std::vector<int2> pairs4; // order 4: every shell pair (c, e), c >= e, in (c, e) order
  int2* d_pairs4 = nullptr;
  size_t mem_budget = 0;    // bytes of shell fields the plan may hold at once (0: no limit)
  int slab_nx = 0;          // > 0: estimates stream x-slabs of this many planes of the evaluation grid
  std::vector<int> zi_off;  // generic Z items of slab k: [zi_off[k], zi_off[k + 1])
  int ngs = 0;              // side of the evaluation grid (<= ng), see choose_eval_grid
  double sum_scale = 1.0;   // (ng / ngs)^3: sums over the ng^3 grid from sums over ngs^3
  double box_len = 0.0, beta = 0.0;
  std::vector<double> edges;
  std::vector<long long> q;       // integer thresholds Q_n
  std::vector<long long> nmodes;  // modes per shell
  std::vector<double> kbar;       // mean |m| per shell
  std::vector<ShellGeom> geom;
  std::vector<bsp_triplet> trips;  // kept bins
  FftStages st_full{}, st_half{};
  int lines_xy = 0, lines_z = 0;
  int n_sm = 0;
  // device buffers
  std::vector<DevBuf> bufs;
  size_t dev_bytes = 0;
  void* tw = nullptr;
  ShellGeom* d_geom = nullptr;
  Item *d_xi = nullptr, *d_yi = nullptr, *d_zi = nullptr;
  int nxi = 0, nyi = 0, nzi = 0;
  void *g1 = nullptr, *g2 = nullptr, *fields = nullptr;
  void* fields32 = nullptr;  // tensor-core plans on the generic passes: FP32 fields before the split
  // tensor-core plans on the warp passes: the Z pass also writes the coarser levels' fields
  TcBin* d_tc_bins = nullptr;  // tensor-core plans: where each kept bin's partial sums are
  ZLevel* d_zlev = nullptr;
  uint32_t* d_zmask = nullptr;
  int n_zlev = 0;
  double* msum = nullptr;
  double* tsum = nullptr;
  int* cell_ptr = nullptr;
  int* cell_idx = nullptr;
  // warp-per-line FP32 passes
  bool warp_fft = false;
  float2 *d_stw = nullptr, *d_stw_half = nullptr;        // stage twiddles, lengths ngs and ngs/2
  float2 *d_stw_ng = nullptr, *d_stw_ng_half = nullptr;  // the same for ng (ball transforms)
  Item *d_wxi = nullptr, *d_wyi = nullptr;
  int nwxi = 0, nwyi = 0;
  int rmax = 0;
  std::vector<ContractLevel> levels;
  // each level's side and bins before split-BF16 plans merge levels (every pair on its smallest
  // exact grid): the algorithm's work, which bsp_plan_stage_work counts
  std::vector<std::pair<int, std::vector<int>>> exact_levels;
  int* d_error = nullptr;
  // gradient resources (built by the first bsp_grad call)
  bool grad_ready = false;
  bool ball_ready = false;
  int adj_np = 0, adj_npairs = 0, adj_entries = 0;
  int2* d_adj_pairs = nullptr;
  int* d_w_ptr = nullptr;
  int* d_w_idx = nullptr;
  double* d_cnorm = nullptr;
  float* d_w = nullptr;
  float* d_gfields = nullptr;      // G_n on the evaluation grid
  void* d_grad_spec = nullptr;     // gradient half spectrum of the ng grid (complex64)
  void* d_tw_ng = nullptr;         // twiddles of the ng grid
  ShellGeom* d_ball = nullptr;     // one pseudo-shell covering every shell's modes
  Item *d_bxi = nullptr, *d_byi = nullptr;
  int nbxi = 0, nbyi = 0;
  void *g1b = nullptr, *g2b = nullptr;
  // per-stage timing (bsp_timing_enable)
  bool timing_on = false;
  int timing_max = 0;
  int timing_calls = 0;
  std::vector<cudaEvent_t> events;   // timing_max x (BSP_N_STAGES + 1)
  long long launches = 0;            // kernels launched by recorded calls
  // host staging for bsp_estimate_host
  void* spec_dev = nullptr;
  double* btrip_dev = nullptr;
  double* bgrid_dev = nullptr;

  size_t elem() const { return prec == BSP_FP64 ? sizeof(double) : sizeof(float); }
  long long nvox() const { return dim == 2 ? (long long)ngs * ngs : (long long)ngs * ngs * ngs; }  // evaluation grid
  int n_groups() const { return (ns + k1_merge - 1) / k1_merge; }
  int n_cells() const { return n_groups() * n_mu * n_t; }
  size_t spec_bytes() const { return (size_t)(dim == 2 ? 1 : ng) * ng * (ng / 2 + 1) * 2 * elem(); }
  size_t field_bytes() const { return (size_t)ns * (size_t)nvox() * elem(); }
  int n_slabs() const { return slab_nx ? (ngs + slab_nx - 1) / slab_nx : 1; }
  int slab_x0(int k) const { return k * slab_nx; }
  int slab_len(int k) const { return slab_nx ? std::min(slab_nx, ngs - k * slab_nx) : ngs; }
  int n_extra() const { return order == 4 ? (int)pairs4.size() : 0; }  // product fields after the ns shells
  int pid4(int c, int e) const { return c * (c + 1) / 2 + e; }         // index of (c, e) in pairs4
  size_t store_bytes() const {                                           // p->fields
    if (dim == 2 || order == 4) return (size_t)(ns + n_extra()) * (size_t)nvox() * elem();
    return (size_t)ns * (size_t)slab_len(0) * ngs * ngs * elem();
  }
};

struct bsp_batch {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n = 0;
};

namespace bsp {

bsp_status dev_alloc(bsp_plan* p, size_t bytes, void** out);
void dev_free(bsp_plan* p, void* d);

template <typename V>
bsp_status dev_upload(bsp_plan* p, const std::vector<V>& h, V** out, cudaStream_t s) {
  void* d = nullptr;
  bsp_status st = dev_alloc(p, h.size() * sizeof(V), &d);
  if (st != BSP_OK) return st;
  if (!h.empty()) BSP_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
  *out = static_cast<V*>(d);
  return BSP_OK;
}

int fft_lines_for(int len, int prec);
void make_items_g(const std::vector<ShellGeom>& geom, int grid, int lines_xy, int lines_z,
                  std::vector<Item>& xi, std::vector<Item>& yi, std::vector<Item>& zi);
void make_items(const bsp_plan* p, int lines_xy, int lines_z, std::vector<Item>& xi,
                std::vector<Item>& yi, std::vector<Item>& zi);
void make_tiles(const std::vector<int>& ta, const std::vector<int>& tb, const std::vector<int>& tc,
                std::vector<int2>& pairs, std::vector<Tile>& tiles, std::vector<int>& map,
                const std::vector<int>* ids = nullptr);
int pick_gridx_n(int n_sm, int ntiles, long long nvox);
// Pair groups of the tensor-core contraction of one level: the slots (f0, f1, f2, flags) of n_tg
// tile groups of kt tiles, and where[i] = (tg * kt + j) * kTcSlots + slot for pair i.
struct TcGrouping {
  int kt = 1;
  int n_tg = 0;
  std::vector<int4> slots;
  std::vector<int> where;
};
TcGrouping group_pairs(const std::vector<int2>& pairs, int nf, int kt_max);
long long g1_elems(const bsp_plan* p);
long long g2_elems(const bsp_plan* p);

// Which passes plan_passes launches: all three over the whole grid, the X and Y passes only, or
// (a value k >= 0) the Z pass of x-slab k, its fields laid out [n][x - x0][y][z] in `fields`.
constexpr int kPassAll = -1;
constexpr int kPassXY = -2;
template <typename T>
bsp_status plan_passes(bsp_plan* p, const void* spec, void* fields, cudaStream_t s, cudaEvent_t* ev,
                       bool split = false, int part = kPassAll);

// The estimate and its stage bookkeeping (bispec_api.cu).
template <typename T>
bsp_status estimate_impl(bsp_plan* p, const void* spec, double* b_trip, double* b_grid, cudaStream_t s);
void stage_work(const bsp_plan* p, double* bytes, double* flops);

}  // namespace bsp
