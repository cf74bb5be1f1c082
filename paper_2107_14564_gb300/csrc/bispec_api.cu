// C ABI of the bispectrum library: plan construction (Sec. 2.1 binning, Eq. (2.10) counts),
// the estimator (Eqs. (2.7)-(2.11)) and the (mu, t) map (Eq. (2.4)).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "common.cuh"

namespace bsp {

// Message of the last failing call on this thread, in a fixed buffer (setting it never
// allocates, so allocation-free entry points can report errors too).
static thread_local char g_error[512];

void set_error_c(const char* msg) {
  size_t n = 0;
  while (msg[n] != 0 && n + 1 < sizeof(g_error)) { g_error[n] = msg[n]; ++n; }
  g_error[n] = 0;
}

void set_error(const std::string& msg) { set_error_c(msg.c_str()); }

bsp_status fail(bsp_status s, const std::string& msg) {
  set_error_c(msg.c_str());
  return s;
}

bsp_status fail_c(bsp_status s, const char* msg) {
  set_error_c(msg);
  return s;
}

bsp_status cuda_fail(cudaError_t e, const char* what) {
  snprintf(g_error, sizeof(g_error), "CUDA error in %s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return BSP_ERR_OOM;
  return BSP_ERR_CUDA;
}

// ---------------------------------------------------------------- host-side helpers
static long long isqrt_ll(long long v) {
  if (v < 0) return -1;
  long long r = (long long)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

// FFT stage list: radix 8 while possible, then 4, 2 and 3.
static bool make_stages(int n, FftStages* st) {
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
  CUtensorMap tmap{};         // tensor-core plans: the level's split fields
  // CUDA-core contraction
  Tile* d_tiles = nullptr;
  int2* d_pairs = nullptr;
  int* d_map = nullptr;       // [ntiles][16] global bin index or -1
  int ntiles = 0, gridx = 0;
  double* partial = nullptr;
  // tensor-core contraction
  int np = 0, mtiles = 0, gridy = 0;
  long long vpb = 0;
  int2* d_tc_pairs = nullptr;
  std::vector<int> tc_off;    // partial-sum entry of each of the level's bins
  int gridy_cap = 0;          // voxel blocks the partial-sum buffer holds
  int tune_mult = 1;          // blocks per M tile / SM count chosen by the autotuner (1 without it)
  double* tc_partial = nullptr;
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

namespace {

bsp_status dev_alloc(bsp_plan* p, size_t bytes, void** out) {
  *out = nullptr;
  if (bytes == 0) bytes = 16;
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(BSP_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
  }
  p->bufs.push_back({d, bytes});
  p->dev_bytes += bytes;
  *out = d;
  return BSP_OK;
}

template <typename V>
bsp_status dev_upload(bsp_plan* p, const std::vector<V>& h, V** out, cudaStream_t s) {
  void* d = nullptr;
  bsp_status st = dev_alloc(p, h.size() * sizeof(V), &d);
  if (st != BSP_OK) return st;
  if (!h.empty()) BSP_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice, s));
  *out = static_cast<V*>(d);
  return BSP_OK;
}

void dev_free(bsp_plan* p, void* d) {
  for (size_t i = 0; i < p->bufs.size(); ++i) {
    if (p->bufs[i].p == d) {
      cudaFree(d);
      p->dev_bytes -= p->bufs[i].bytes;
      p->bufs.erase(p->bufs.begin() + i);
      return;
    }
  }
}

int fft_lines_for(int len, int prec) {
  const int e = prec == BSP_FP64 ? FftElems<double>::value : FftElems<float>::value;
  int l = e * kFftThreads / len;
  return l < 1 ? 1 : l;
}

// Work items of the three passes for shells `geom` on a grid of side `grid`.
void make_items_g(const std::vector<ShellGeom>& geom, int grid, int lines_xy, int lines_z,
                  std::vector<Item>& xi, std::vector<Item>& yi, std::vector<Item>& zi) {
  const int ng = grid;
  xi.clear(); yi.clear(); zi.clear();
  for (int n = 0; n < (int)geom.size(); ++n) {
    const ShellGeom& g = geom[n];
    const int r = g.r;
    for (int ky = -(r - 1); ky <= r - 1; ++ky) {
      const long long rem = (long long)g.qhi - 1 - (long long)ky * ky;
      const int kzmax = (int)isqrt_ll(rem) + 1;  // kz with ky^2 + kz^2 < qhi
      for (int kz0 = 0; kz0 < kzmax; kz0 += lines_xy)
        xi.push_back({n, ky, kz0, std::min(lines_xy, kzmax - kz0)});
    }
    for (int x = 0; x < ng; ++x)
      for (int kz0 = 0; kz0 < r; kz0 += lines_xy) yi.push_back({n, x, kz0, std::min(lines_xy, r - kz0)});
    for (int x = 0; x < ng; ++x)
      for (int y0 = 0; y0 < ng; y0 += lines_z) zi.push_back({n, x, y0, std::min(lines_z, ng - y0)});
  }
}

void make_items(const bsp_plan* p, int lines_xy, int lines_z, std::vector<Item>& xi,
                std::vector<Item>& yi, std::vector<Item>& zi) {
  if (p->dim == 2) {  // 2D rings: k_y lines for the X pass (xi), x rows for the C2R along y (zi)
    xi.clear(); yi.clear(); zi.clear();
    for (int n = 0; n < p->ns; ++n) {
      const int r = p->geom[n].r;
      for (int ky0 = 0; ky0 < r; ky0 += lines_xy) xi.push_back({n, 0, ky0, std::min(lines_xy, r - ky0)});
      for (int x0 = 0; x0 < p->ngs; x0 += lines_z) zi.push_back({n, 0, x0, std::min(lines_z, p->ngs - x0)});
    }
    return;
  }
  make_items_g(p->geom, p->ngs, lines_xy, lines_z, xi, yi, zi);
}

// Tiles of up to 4 consecutive pairs x 4 consecutive c over a list of bins sorted by (a, b, c).
void make_tiles(const std::vector<int>& ta, const std::vector<int>& tb, const std::vector<int>& tc,
                std::vector<int2>& pairs, std::vector<Tile>& tiles, std::vector<int>& map,
                const std::vector<int>* ids = nullptr) {
  pairs.clear(); tiles.clear(); map.clear();
  std::vector<std::vector<std::pair<int, int>>> pc;  // per pair: (c, bin)
  for (size_t t = 0; t < ta.size(); ++t) {
    if (pairs.empty() || pairs.back().x != ta[t] || pairs.back().y != tb[t]) {
      pairs.push_back(make_int2(ta[t], tb[t]));
      pc.emplace_back();
    }
    pc.back().push_back({tc[t], ids ? (*ids)[t] : (int)t});
  }
  const int np = (int)pairs.size();
  for (int p0 = 0; p0 < np; p0 += 4) {
    const int cnt = std::min(4, np - p0);
    int cmin = 1 << 30, cmax = -1;
    for (int i = 0; i < cnt; ++i)
      for (auto& e : pc[p0 + i]) { cmin = std::min(cmin, e.first); cmax = std::max(cmax, e.first); }
    for (int c0 = cmin - cmin % 4; c0 <= cmax; c0 += 4) {
      int m[16];
      bool any = false;
      for (int k = 0; k < 16; ++k) m[k] = -1;
      for (int i = 0; i < cnt; ++i)
        for (auto& e : pc[p0 + i])
          if (e.first >= c0 && e.first < c0 + 4) { m[i * 4 + (e.first - c0)] = e.second; any = true; }
      if (!any) continue;
      tiles.push_back({p0, cnt, c0, 0});
      for (int k = 0; k < 16; ++k) map.push_back(m[k]);
    }
  }
}

// Rows of the tensor-core contraction: pair i goes to row row_of[i]. Every row costs the same
// generation work, so pairs are packed densely; their order only matters for shared-memory bank
// conflicts. A generator thread reads 16 bytes of field a and of field b of its row per load, and
// a 128-bit load is served in four phases of 8 consecutive lanes; field n's 16 bytes sit in bank
// group n mod 8 of their 128-byte line (the TMA's swizzle), so a phase is conflict-free when its
// distinct a take distinct values mod 8, and its distinct b too. Rows are filled 8 at a time by
// first fit over the pairs in (a, b) order. Padding rows of a phase repeat its first pair, encoded
// as (-a - 1, -b - 1) (a broadcast, never read back). Returns the number of rows (multiple of 8).
int assign_tc_rows(const std::vector<int2>& pairs, std::vector<int>& row_of, std::vector<int2>& rows) {
  row_of.assign(pairs.size(), -1);
  rows.clear();
  std::vector<int> pending(pairs.size());
  for (size_t i = 0; i < pairs.size(); ++i) pending[i] = (int)i;
  while (!pending.empty()) {
    int a_at[8], b_at[8];
    for (int k = 0; k < 8; ++k) a_at[k] = b_at[k] = -1;
    std::vector<int> take, rest;
    for (int i : pending) {
      const int a = pairs[i].x, b = pairs[i].y;
      const bool fit = take.size() < 8 && (a_at[a & 7] < 0 || a_at[a & 7] == a) && (b_at[b & 7] < 0 || b_at[b & 7] == b);
      if (fit) {
        a_at[a & 7] = a;
        b_at[b & 7] = b;
        take.push_back(i);
      } else {
        rest.push_back(i);
      }
    }
    for (int i : take) {
      row_of[i] = (int)rows.size();
      rows.push_back(pairs[i]);
    }
    const int2 first = pairs[take[0]];
    while (rows.size() % 8 != 0) rows.push_back(make_int2(-first.x - 1, -first.y - 1));
    pending.swap(rest);
  }
  return (int)rows.size();
}

// Shell fields of one precision: X, Y, Z passes for every shell.
template <typename T>
bsp_status run_passes(const bsp_plan* p, const void* spec, int rsd, void* tw, void* g1, void* g2,
                      void* fields, const Item* xi, int nxi, const Item* yi, int nyi, const Item* zi,
                      int nzi, int lines_xy, int lines_z, cudaStream_t s, int kweight = 0, bool do_xy = true,
                      bool do_z = true, int slab_x0 = 0, int slab_nx = 0) {
  PassArgs a{};
  a.n_sm = p->n_sm;
  a.kweight = kweight;
  a.spec = spec;
  a.g1 = g1;
  a.g2 = g2;
  a.fields = fields;
  a.tw = tw;
  a.geom = p->d_geom;
  a.ng = p->ng;
  a.ngs = p->ngs;
  a.rsd = rsd;
  a.beta = p->beta;
  bsp_status st;
  if (p->dim == 2) {  // 2D rings: X pass, then the C2R along y (the Z-pass kernel on its rows)
    a.st = p->st_full;
    a.items = xi;
    if ((st = launch_ring_xpass<T>(a, nxi, lines_xy, s)) != BSP_OK) return st;
    a.items = zi;
    a.st = p->st_half;
    a.g2 = g1;
    a.slab_x0 = 0;
    a.slab_nx = 1;
    return launch_zpass<T>(a, nzi, lines_z, s);
  }
  if (do_xy) {
    a.st = p->st_full;
    a.items = xi;
    st = launch_xpass<T>(a, nxi, lines_xy, s);
    if (st != BSP_OK) return st;
    a.items = yi;
    st = launch_ypass<T>(a, nyi, lines_xy, s);
    if (st != BSP_OK) return st;
  }
  if (!do_z) return BSP_OK;
  a.items = zi;
  a.st = p->st_half;
  a.slab_x0 = slab_x0;
  a.slab_nx = slab_nx;
  return launch_zpass<T>(a, nzi, lines_z, s);
}

int pick_gridx_n(int n_sm, int ntiles, long long nvox) {
  const int gy = (ntiles + 255) / 256;
  int gx = (4 * n_sm) / std::max(gy, 1);
  gx = std::max(gx, 1);
  const long long chunks = (nvox + 63) / 64;
  if (gx > chunks) gx = (int)chunks;
  return gx;
}

int pick_gridx(const bsp_plan* p, int ntiles) { return pick_gridx_n(p->n_sm, ntiles, p->nvox()); }

bsp_status validate(const bsp_plan_desc* d) {
  if (!d) return fail(BSP_ERR_INVALID_ARG, "desc is NULL");
  if (d->dim != 0 && d->dim != 2 && d->dim != 3) return fail(BSP_ERR_INVALID_ARG, "dim must be 0, 2 or 3");
  if (d->order != 0 && d->order != 3 && d->order != 4) return fail(BSP_ERR_INVALID_ARG, "order must be 0, 3 or 4");
  if (d->order == 4) {
    if (d->precision == BSP_MIXED_BF16X3 || d->n_shells > 16 || d->label_k != BSP_LABEL_SHELL_MEAN || d->mem_budget_bytes)
      return fail(BSP_ERR_NOT_SUPPORTED, "order 4: FP64 or FP32, at most 16 shells, shell-mean labels, no memory budget");
    if (d->n_mu != 1 || d->n_t != 1) return fail(BSP_ERR_INVALID_ARG, "order 4: n_mu = n_t = 1");
  }
  if (d->dim == 2) {
    if (d->ng < 16 || d->ng > 4096 || (d->ng % 2) != 0)
      return fail(BSP_ERR_NOT_SUPPORTED, "2D: ng must be even and within [16, 4096]");
    if (d->precision == BSP_MIXED_BF16X3 || d->rsd || d->label_k != BSP_LABEL_SHELL_MEAN || d->mem_budget_bytes)
      return fail(BSP_ERR_NOT_SUPPORTED, "2D plans: FP64 or FP32, no RSD, shell-mean labels, no memory budget");
  } else if (d->ng < 16 || d->ng > 1024 || (d->ng % 2) != 0) {
    return fail(BSP_ERR_NOT_SUPPORTED, "ng must be even and within [16, 1024]");
  }
  FftStages st;
  if (!make_stages(d->ng, &st) || !make_stages(d->ng / 2, &st))
    return fail(BSP_ERR_NOT_SUPPORTED, "ng must be a product of 2s and 3s");
  if (!(d->box_len > 0.0) || !isfinite(d->box_len)) return fail(BSP_ERR_INVALID_ARG, "box_len must be > 0");
  if (d->n_shells < 1 || d->n_shells > 256) return fail(BSP_ERR_INVALID_ARG, "n_shells out of range");
  if (!d->edges_kf) return fail(BSP_ERR_INVALID_ARG, "edges_kf is NULL");
  for (int i = 0; i <= d->n_shells; ++i)
    if (!isfinite(d->edges_kf[i]) || d->edges_kf[i] < 0.0) return fail(BSP_ERR_INVALID_ARG, "bad edge");
  for (int i = 0; i < d->n_shells; ++i)
    if (!(d->edges_kf[i + 1] > d->edges_kf[i])) return fail(BSP_ERR_INVALID_ARG, "edges must increase");
  if (d->k1_merge < 0) return fail(BSP_ERR_INVALID_ARG, "k1_merge must be >= 0");
  if (d->label_k != BSP_LABEL_SHELL_MEAN && d->label_k != BSP_LABEL_TRIANGLE_MEAN)
    return fail(BSP_ERR_INVALID_ARG, "label_k must be a bsp_label_k");
  if (d->n_mu < 1 || d->n_t < 1 || d->n_mu > 4096 || d->n_t > 4096)
    return fail(BSP_ERR_INVALID_ARG, "n_mu and n_t must be >= 1");
  if (d->precision < BSP_FP64 || d->precision > BSP_MIXED_BF16X3)
    return fail(BSP_ERR_INVALID_ARG, "unknown precision");
  if (d->rsd != 0 && d->rsd != 1) return fail(BSP_ERR_INVALID_ARG, "rsd must be 0 or 1");
  if (d->precision == BSP_MIXED_BF16X3 && (d->ng % 8 != 0 || d->n_shells > 64))
    return fail(BSP_ERR_NOT_SUPPORTED, "BSP_MIXED_BF16X3 needs ng % 8 == 0 and at most 64 shells");
  if (d->rsd && !isfinite(d->beta)) return fail(BSP_ERR_INVALID_ARG, "beta must be finite");
  return BSP_OK;
}

// The evaluation grid. Every shell mode has |m_i| <= r_max - 1, so a triple product of three shell
// fields only holds wavevectors with |k_i| <= 3 (r_max - 1). Summing it over any grid of side
// S > 3 (r_max - 1) keeps only k = 0, exactly as the ng^3 grid does (the argument of Eq. (2.6) and
// of the cap after Eq. (2.12)): sum over ng^3 = (ng / S)^3 sum over S^3, and the shell fields
// sampled on the S grid are the same band-limited functions. The plan evaluates fields and
// triple products on the smallest such S it has kernels for (at most ng). A product of p fields
// (order-p plans) needs S > p (r_max - 1) by the same argument.
bool fft_size_ok(int n) {
  if (n < 16 || n % 8 != 0) return false;
  int m = n;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

void choose_eval_grid(bsp_plan* p) {
  int rmax = 0;
  for (int n = 0; n < p->ns; ++n) rmax = std::max(rmax, (int)isqrt_ll(p->q[n + 1] - 1) + 1);
  const int need = p->order * (rmax - 1) + 1;  // S >= need (a product of `order` fields)
  int best = p->ng;
  for (int sz = 16; sz < p->ng; ++sz) {
    if (sz < need || !fft_size_ok(sz)) continue;
    // FP32 plans prefer the sizes the warp-per-line kernels handle
    if (p->dim == 3 && p->prec != BSP_FP64 && p->ng >= 128 && !warp_fft_supported(sz)) continue;
    best = sz;
    break;
  }
  p->ngs = best;
  const double f = (double)p->ng / (double)p->ngs;
  p->sum_scale = p->dim == 2 ? f * f : f * f * f;
}

// Host part of the plan (Sec. 2.1): thresholds, cap, mode counts, means, geometry.
bsp_status host_plan(bsp_plan* p, const bsp_plan_desc* d) {
  p->ng = d->ng;
  p->ns = d->n_shells;
  p->n_mu = d->n_mu;
  p->n_t = d->n_t;
  p->rsd = d->rsd;
  p->beta = d->rsd ? d->beta : 0.0;
  p->prec = d->precision;
  p->autotune = d->autotune;
  p->k1_merge = d->k1_merge > 1 ? d->k1_merge : 1;
  p->label_k = d->label_k;
  p->dim = d->dim == 2 ? 2 : 3;
  p->order = d->order == 4 ? 4 : 3;
  p->box_len = d->box_len;
  p->edges.assign(d->edges_kf, d->edges_kf + d->n_shells + 1);
  p->q.resize(p->ns + 1);
  for (int n = 0; n <= p->ns; ++n) {
    const double e = p->edges[n];
    p->q[n] = (long long)ceil(e * e);
  }
  p->q[0] = std::max(1LL, p->q[0]);
  for (int n = 0; n < p->ns; ++n)
    if (p->q[n + 1] <= p->q[n]) return fail(BSP_ERR_INVALID_ARG, "shell " + std::to_string(n) + " is empty");
  const long long qmax = p->q[p->ns];
  // cap after Eq. (2.12): every mode |m| < Ng/3  <=>  9 (Q_Ns - 1) < Ng^2; Ng / p for the
  // order-p sum (Sec. 4)
  if ((long long)p->order * p->order * (qmax - 1) >= (long long)p->ng * p->ng)
    return fail(BSP_ERR_ALIASING, "largest shell reaches k >= 2 pi Ng / (" + std::to_string(p->order) + " L)");
  // mode counts per |m|^2
  const long long rr = isqrt_ll(qmax - 1);
  std::vector<long long> cnt(qmax, 0);
  for (long long x = -rr; x <= rr; ++x)
    for (long long y = -rr; y <= rr; ++y) {
      const long long qxy = x * x + y * y;
      if (qxy >= qmax) continue;
      if (p->dim == 2) {  // rings: modes of the plane
        cnt[qxy] += 1;
        continue;
      }
      for (long long z = -rr; z <= rr; ++z) {
        const long long qq = qxy + z * z;
        if (qq < qmax) cnt[qq] += 1;
      }
    }
  p->nmodes.assign(p->ns, 0);
  p->kbar.assign(p->ns, 0.0);
  for (int n = 0; n < p->ns; ++n) {
    double s = 0.0;
    long long c = 0;
    for (long long qq = p->q[n]; qq < p->q[n + 1]; ++qq) {
      if (cnt[qq]) {
        s += (double)cnt[qq] * sqrt((double)qq);
        c += cnt[qq];
      }
    }
    if (c == 0) return fail(BSP_ERR_INVALID_ARG, "shell " + std::to_string(n) + " holds no modes");
    p->nmodes[n] = c;
    p->kbar[n] = s / (double)c;
  }
  choose_eval_grid(p);
  make_stages(p->ngs, &p->st_full);
  make_stages(p->ngs / 2, &p->st_half);
  // geometry: complex offsets of each shell in the X and Y pass buffers
  p->geom.resize(p->ns);
  long long o1 = 0, o2 = 0;
  for (int n = 0; n < p->ns; ++n) {
    ShellGeom& g = p->geom[n];
    g.qlo = (int)p->q[n];
    g.qhi = (int)p->q[n + 1];
    g.r = (int)isqrt_ll(p->q[n + 1] - 1) + 1;
    g.pad = 0;
    g.g1_off = o1;
    g.g2_off = o2;
    if (p->dim == 2) {  // one buffer of X-pass rows [x][k_y < r], read again by the C2R along y
      g.g2_off = o1;
      o1 += (long long)p->ngs * g.r;
      continue;
    }
    o1 += (long long)p->ngs * (2 * g.r - 1) * g.r;
    o2 += (long long)p->ngs * p->ngs * g.r;
  }
  // memory budget: stream x-slabs of the evaluation grid when all fields do not fit
  p->mem_budget = d->mem_budget_bytes;
  if (p->mem_budget > 0 && p->mem_budget < p->field_bytes()) {
    if (p->prec == BSP_MIXED_BF16X3)
      return fail(BSP_ERR_NOT_SUPPORTED, "mem_budget_bytes below the shell fields of a split-BF16 plan");
    const size_t plane = (size_t)p->ns * p->ngs * p->ngs * p->elem();
    if (p->mem_budget < plane) return fail(BSP_ERR_INVALID_ARG, "mem_budget_bytes below one x-plane of all shell fields");
    p->slab_nx = (int)std::min<size_t>(p->mem_budget / plane, (size_t)p->ngs - 1);
  }
  return BSP_OK;
}

// Generic Z-pass items reordered slab by slab (x-slabs of slab_nx planes; one slab when 0), with
// the start of each slab's range in off[k].
void slab_items(int slab_nx, int grid, std::vector<Item>& zi, std::vector<int>& off) {
  const int nsl = slab_nx ? (grid + slab_nx - 1) / slab_nx : 1;
  std::vector<Item> out;
  off.assign(nsl + 1, 0);
  for (int k = 0; k < nsl; ++k) {
    for (const Item& it : zi)
      if (!slab_nx || it.u / slab_nx == k) out.push_back(it);
    off[k + 1] = (int)out.size();
  }
  zi.swap(out);
}

long long g1_elems(const bsp_plan* p) {
  const ShellGeom& g = p->geom.back();
  if (p->dim == 2) return g.g1_off + (long long)p->ngs * g.r;  // 2D X-pass rows [x][k_y < r]
  return g.g1_off + (long long)p->ngs * (2 * g.r - 1) * g.r;
}
long long g2_elems(const bsp_plan* p) {
  const ShellGeom& g = p->geom.back();
  if (p->dim == 2) return 1;  // unused by 2D plans
  return g.g2_off + (long long)p->ngs * p->ngs * g.r;
}

// Contraction autotuner (plans created with autotune = 1): for every tensor-core level, time its
// kernel on the plan's own buffers with the voxel range of each M tile split over m x (SM count)
// blocks, m in kTuneMults (fewer when the level has fewer 128-voxel chunks), 3 launches after one
// warm-up each, and keep the fastest split. More blocks than SMs trade partial sums and block
// start-up for a shorter tail. The values computed are the same for every split up to the
// order of the FP64 cross-block sums.
bsp_status autotune_levels(bsp_plan* p, cudaStream_t s) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BSP_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(ce, "cudaEventCreate"); }
  bsp_status st = BSP_OK;
  for (ContractLevel& L : p->levels) {
    if (L.mtiles == 0) continue;
    const long long chunks = L.nvox() / kTcVoxelChunk;
    float best = 1e30f;
    long long best_vpb = L.vpb;
    int best_gy = L.gridy, best_m = 1;
    for (int t = 0; t < kNumTune && st == BSP_OK; ++t) {
      const long long gy = std::min<long long>((long long)kTuneMults[t] * std::max(1, p->n_sm), chunks);
      const long long vpb = ((chunks + gy - 1) / gy) * kTcVoxelChunk;
      const int gridy = (int)((L.nvox() + vpb - 1) / vpb);
      if (gridy > L.gridy_cap && gridy > L.gridy) continue;
      TcArgs a{};
      a.nvox = L.nvox();
      a.ns = (int)L.shells.size();
      a.np = L.np;
      a.pair_ab = L.d_tc_pairs;
      a.n_mtiles = L.mtiles;
      a.gridy = gridy;
      a.vox_per_block = vpb;
      a.partial = L.tc_partial;
      a.error = p->d_error;
      if ((st = launch_contract_tc(a, &L.tmap, s)) != BSP_OK) break;
      if ((ce = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(ce, "cudaEventRecord"); break; }
      for (int r = 0; r < 3 && st == BSP_OK; ++r) st = launch_contract_tc(a, &L.tmap, s);
      if (st != BSP_OK) break;
      if ((ce = cudaEventRecord(e1, s)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(ce, "autotune timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_vpb = vpb; best_gy = gridy; best_m = kTuneMults[t]; }
    }
    L.vpb = best_vpb;
    L.gridy = best_gy;
    L.tune_mult = best_m;
    if (st != BSP_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

// FFT pass autotuner (plans created with autotune = 1 on the warp passes): the persistent Y and Z
// passes are timed on the plan's own buffers (a zero spectrum; the work does not depend on the
// values) with grids of 1, 2, 3, 4, 6, 8, 12 and 16 x (SM count) blocks and as many as fit, 3 launches
// after one warm-up each, and the fastest grid is kept. The grid changes only which block takes
// which lines, not what any line computes.
// Which passes plan_passes launches: all three over the whole grid, the X and Y passes only, or
// (a value k >= 0) the Z pass of x-slab k, its fields laid out [n][x - x0][y][z] in `fields`.
constexpr int kPassAll = -1;
constexpr int kPassXY = -2;
template <typename T>
bsp_status plan_passes(bsp_plan* p, const void* spec, void* fields, cudaStream_t s, cudaEvent_t* ev,
                       bool split = false, int part = kPassAll);
bsp_status autotune_passes(bsp_plan* p, cudaStream_t s) {
  if (!p->warp_fft) return BSP_OK;
  void* spec = nullptr;
  bsp_status st = dev_alloc(p, p->spec_bytes(), &spec);
  if (st != BSP_OK) return st;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaMemsetAsync(spec, 0, p->spec_bytes(), s);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) st = cuda_fail(ce, "pass autotuner setup");
  const bool split = p->prec == BSP_MIXED_BF16X3;
  const int mults[] = {0, 1, 2, 3, 4, 6, 8, 12, 16};  // 0: as many as fit
  int* knob[2] = {&p->y_blocks, &p->z_blocks};
  for (int pass = 0; pass < 2 && st == BSP_OK; ++pass) {
    float best = 1e30f;
    int best_blocks = 0;
    for (int m : mults) {
      *knob[pass] = m * p->n_sm;
      // warm-up (the Y pass needs the X pass output once; the Z pass reads what Y wrote)
      if ((st = plan_passes<float>(p, spec, p->fields, s, nullptr, split, kPassAll)) != BSP_OK) break;
      if ((ce = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(ce, "cudaEventRecord"); break; }
      for (int r = 0; r < 3 && st == BSP_OK; ++r) st = plan_passes<float>(p, spec, p->fields, s, nullptr, split, kPassAll);
      if (st != BSP_OK) break;
      if ((ce = cudaEventRecord(e1, s)) != cudaSuccess || (ce = cudaEventSynchronize(e1)) != cudaSuccess) {
        st = cuda_fail(ce, "pass autotune timing");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_blocks = *knob[pass]; }
    }
    *knob[pass] = best_blocks;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  dev_free(p, spec);
  return st;
}

// Contraction levels (see ContractLevel): each pair (a, b) of the kept bins goes to the smallest
// divisor g of the evaluation grid (g % 8 == 0, g >= 16) above r_a + r_b + r_cmax - 3, the largest
// wavevector component of its triple products.
bsp_status build_levels(bsp_plan* p, cudaStream_t s) {
  const int S = p->ngs;
  std::vector<std::pair<int, std::vector<int>>> by_g;  // ascending g
  auto bins_of = [&](int g) -> std::vector<int>& {
    for (auto& e : by_g)
      if (e.first == g) return e.second;
    by_g.push_back({g, {}});
    return by_g.back().second;
  };
  size_t t = 0;
  while (t < p->trips.size()) {
    size_t u = t;
    int cmax = 0;
    while (u < p->trips.size() && p->trips[u].a == p->trips[t].a && p->trips[u].b == p->trips[t].b) {
      cmax = std::max(cmax, p->trips[u].c);
      ++u;
    }
    const int need = p->geom[p->trips[t].a].r + p->geom[p->trips[t].b].r + p->geom[cmax].r - 2;
    int g = S;
    for (int cand = 16; cand < S && !p->slab_nx && p->dim == 3 && p->order == 3; cand += 8)  // else one level
      if (S % cand == 0 && cand >= need) { g = cand; break; }
    std::vector<int>& v = bins_of(g);
    for (size_t w = t; w < u; ++w) v.push_back((int)w);
    t = u;
  }
  std::sort(by_g.begin(), by_g.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  const size_t re = p->elem();
  bsp_status st;
  std::vector<ZLevel> zl;  // levels the split Z pass writes
  std::vector<int> zt;     // their strides
  for (auto& e : by_g) {
    ContractLevel L;
    L.dim = p->dim;
    L.g = e.first;
    L.stride = S / L.g;
    const double f = (double)p->ng / (double)L.g;
    L.scale = p->dim == 2 ? f * f : f * f * f;
    L.top = L.g == S;
    L.bins = e.second;
    std::vector<int> loc(p->ns, -1);
    if (L.top) {
      for (int n = 0; n < p->ns; ++n) { L.shells.push_back(n); loc[n] = n; }
      for (int j = 0; j < p->n_extra(); ++j) L.shells.push_back(p->ns + j);  // order 4: pair products
    } else {
      std::vector<char> used(p->ns, 0);
      for (int b : L.bins) used[p->trips[b].a] = used[p->trips[b].b] = used[p->trips[b].c] = 1;
      for (int n = 0; n < p->ns; ++n)
        if (used[n]) { loc[n] = (int)L.shells.size(); L.shells.push_back(n); }
    }
    const int nsh = (int)L.shells.size();
    std::vector<int> la, lb, lc;
    for (int b : L.bins) {
      const bsp_triplet& t = p->trips[b];
      la.push_back(loc[t.a]);
      lb.push_back(loc[t.b]);
      lc.push_back(p->order == 4 ? p->ns + p->pid4(t.c, t.e) : loc[t.c]);  // order 4: top level only
    }
    std::vector<int2> pairs;
    std::vector<Tile> tiles;
    std::vector<int> map;
    make_tiles(la, lb, lc, pairs, tiles, map, &L.bins);
    void* tmp = nullptr;
    if (p->prec == BSP_MIXED_BF16X3) {
      L.np = tc_padded_shells(nsh);
      std::vector<int> row_of;
      std::vector<int2> rows;
      const int nrows = assign_tc_rows(pairs, row_of, rows);
      L.mtiles = (nrows + 127) / 128;
      // 8-row phases dealt round-robin over the M tiles, so every tile has the same work
      const int mt = std::max(L.mtiles, 1);
      auto place = [mt](int r) { const int ph = r / 8; return (ph % mt) * 128 + (ph / mt) * 8 + r % 8; };
      std::vector<int2> pab((size_t)mt * 128, make_int2(-1, -1));
      for (int i = 0; i < nrows; ++i) pab[place(i)] = rows[i];
      for (int& r : row_of) r = place(r);
      std::vector<int> tmap(L.bins.size());
      int pi = -1;
      for (size_t i = 0; i < L.bins.size(); ++i) {
        if (i == 0 || la[i] != la[i - 1] || lb[i] != lb[i - 1]) ++pi;
        tmap[i] = row_of[pi] * L.np + lc[i];
      }
      const long long chunks = L.nvox() / kTcVoxelChunk;
      long long gy = std::min<long long>(std::max(1, p->n_sm), chunks);
      L.vpb = ((chunks + gy - 1) / gy) * kTcVoxelChunk;
      L.gridy = (int)((L.nvox() + L.vpb - 1) / L.vpb);
      // partial sums sized for the largest split the autotuner may pick
      const long long gmax = p->autotune ? std::min<long long>((long long)kTuneMults[kNumTune - 1] * std::max(1, p->n_sm), chunks) : gy;
      L.gridy_cap = (int)((L.nvox() + ((chunks + gmax - 1) / gmax) * kTcVoxelChunk - 1) / (((chunks + gmax - 1) / gmax) * kTcVoxelChunk));
      if ((st = dev_upload(p, pab, &L.d_tc_pairs, s)) != BSP_OK) return st;
      L.tc_off = tmap;
      if ((st = dev_alloc(p, tc_partial_doubles(std::max(L.mtiles, 1), std::max(L.gridy, L.gridy_cap), L.np) * sizeof(double), &tmp)) != BSP_OK)
        return st;
      L.tc_partial = static_cast<double*>(tmp);
    } else {
      L.ntiles = (int)tiles.size();
      L.gridx = pick_gridx_n(p->n_sm, L.ntiles, L.nvox());
      if ((st = dev_upload(p, tiles, &L.d_tiles, s)) != BSP_OK) return st;
      if ((st = dev_upload(p, pairs, &L.d_pairs, s)) != BSP_OK) return st;
      if ((st = dev_upload(p, map, &L.d_map, s)) != BSP_OK) return st;
      if ((st = dev_alloc(p, (size_t)std::max(L.gridx, 1) * std::max(L.ntiles, 1) * 16 * sizeof(double), &tmp)) != BSP_OK)
        return st;
      L.partial = static_cast<double*>(tmp);
    }
    if (!L.top) {
      std::vector<int> src = L.shells;
      if (p->prec == BSP_MIXED_BF16X3)  // split planes: high parts, then low parts (ns planes later)
        for (int n : L.shells) src.push_back(p->ns + n);
      if ((st = dev_upload(p, src, &L.d_shells, s)) != BSP_OK) return st;
      if ((st = dev_alloc(p, (size_t)nsh * (size_t)L.nvox() * re, &L.fields)) != BSP_OK) return st;
    }
    if (p->prec == BSP_MIXED_BF16X3 && L.mtiles > 0) {
      st = encode_split_map(&L.tmap, L.top ? p->fields : L.fields, L.nvox(), nsh, L.np);
      if (st != BSP_OK) return st;
    }
    if (p->prec == BSP_MIXED_BF16X3 && p->warp_fft && !L.top) {
      ZLevel z{};
      z.dst = static_cast<uint16_t*>(L.fields);
      z.lo_off = (long long)nsh * L.nvox();
      int* dloc = nullptr;
      if ((st = dev_upload(p, loc, &dloc, s)) != BSP_OK) return st;
      z.loc = dloc;
      z.g = L.g;
      z.t = L.stride;
      z.rt = 1.0f / (float)L.stride;
      zl.push_back(z);
      zt.push_back(L.stride);
    }
    p->levels.push_back(std::move(L));
  }
  if (p->prec == BSP_MIXED_BF16X3 && p->autotune) {
    if ((st = autotune_levels(p, s)) != BSP_OK) return st;
  }
  if (p->prec == BSP_MIXED_BF16X3) {
    std::vector<TcBin> tb(p->trips.size());
    for (const ContractLevel& L : p->levels)
      for (size_t i = 0; i < L.bins.size(); ++i) {
        TcBin& b = tb[L.bins[i]];
        b.partial = L.tc_partial;
        b.stride = (long long)L.mtiles * 128 * L.np;
        b.gridy = L.gridy;
        b.off = L.tc_off[i];
        b.scale = L.scale;
      }
    if ((st = dev_upload(p, tb, &p->d_tc_bins, s)) != BSP_OK) return st;
  }
  if (!zl.empty()) {
    if (zl.size() > 32) return fail(BSP_ERR_NOT_SUPPORTED, "more than 32 contraction levels");
    std::vector<uint32_t> mask(S, 0u);
    for (int i = 0; i < S; ++i)
      for (size_t l = 0; l < zt.size(); ++l)
        if (i % zt[l] == 0) mask[i] |= 1u << l;
    if ((st = dev_upload(p, zl, &p->d_zlev, s)) != BSP_OK) return st;
    if ((st = dev_upload(p, mask, &p->d_zmask, s)) != BSP_OK) return st;
    p->n_zlev = (int)zl.size();
  }
  return BSP_OK;
}

// FP64 sums over the evaluation grid (unscaled) of products of three counting fields, Eq. (2.10):
// indices n < ns name i_n of Eq. (2.11); with `lengths`, indices ns + n name the length-weighted
// counting field w_n = sum_{k in n} |k| e^{i k.x} (|k| in units of k_f). Triplets that share
// their first two indices should be adjacent. out[ids ? ids[t] : t] = the sum of triplet t.
bsp_status plan_sums(bsp_plan* p, bool lengths, const std::vector<int>& ca, const std::vector<int>& cb,
                     const std::vector<int>& cc, const std::vector<int>* ids, std::vector<double>& tsum,
                     cudaStream_t s) {
  const int nf = lengths ? 2 * p->ns : p->ns + p->n_extra();  // order 4: shell fields, then pair products
  const int S = p->ngs;
  const int lxy = fft_lines_for(S, BSP_FP64);
  const int lz = fft_lines_for(S / 2, BSP_FP64);
  std::vector<Item> xi, yi, zi;
  make_items(p, lxy, lz, xi, yi, zi);
  // under a memory budget the FP64 fields are produced and contracted one x-slab at a time
  int nx = S;
  if (p->mem_budget > 0) {
    const size_t plane = (size_t)nf * S * S * sizeof(double);
    nx = (int)std::max<size_t>(1, std::min<size_t>((size_t)S, p->mem_budget / plane));
  }
  const int slab = nx < S ? nx : 0;
  std::vector<int> zoff;
  slab_items(slab, S, zi, zoff);
  const int nsl = (int)zoff.size() - 1;
  const long long slab_vox = p->dim == 2 ? (long long)S * S : (long long)nx * S * S;
  std::vector<void*> tmp;
  auto cleanup = [&]() {
    cudaStreamSynchronize(s);
    for (void* d : tmp) dev_free(p, d);
  };
  void *tw = nullptr, *g1 = nullptr, *g2 = nullptr, *g2w = nullptr, *f = nullptr;
  Item *dxi = nullptr, *dyi = nullptr, *dzi = nullptr;
  bsp_status st;
#define TRY(x) do { st = (x); if (st != BSP_OK) { cleanup(); return st; } } while (0)
  TRY(dev_alloc(p, S * sizeof(double2), &tw)); tmp.push_back(tw);
  TRY(dev_alloc(p, g1_elems(p) * sizeof(double2), &g1)); tmp.push_back(g1);
  TRY(dev_alloc(p, g2_elems(p) * sizeof(double2), &g2)); tmp.push_back(g2);
  if (slab && lengths) { TRY(dev_alloc(p, g2_elems(p) * sizeof(double2), &g2w)); tmp.push_back(g2w); }
  TRY(dev_alloc(p, (size_t)nf * slab_vox * sizeof(double), &f)); tmp.push_back(f);
  TRY(dev_upload(p, xi, &dxi, s)); tmp.push_back(dxi);
  TRY(dev_upload(p, yi, &dyi, s)); tmp.push_back(dyi);
  TRY(dev_upload(p, zi, &dzi, s)); tmp.push_back(dzi);
  TRY(launch_twiddles<double>(tw, S, s));
  if (!slab) {
    TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2, f, dxi, (int)xi.size(), dyi, (int)yi.size(), dzi,
                           (int)zi.size(), lxy, lz, s));
    if (p->order == 4)
      TRY(launch_pair_fields<double>(f, slab_vox, p->d_pairs4, p->n_extra(),
                                     static_cast<double*>(f) + (size_t)p->ns * slab_vox, p->n_sm, s));
    if (lengths)
      TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2, static_cast<double*>(f) + (size_t)p->ns * slab_vox,
                             dxi, (int)xi.size(), dyi, (int)yi.size(), dzi, (int)zi.size(), lxy, lz, s, 1));
  } else {
    TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2, f, dxi, (int)xi.size(), dyi, (int)yi.size(), dzi, 0, lxy,
                           lz, s, 0, true, false));
    if (lengths)
      TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2w, f, dxi, (int)xi.size(), dyi, (int)yi.size(), dzi, 0, lxy,
                             lz, s, 1, true, false));
  }
  std::vector<int2> pairs;
  std::vector<Tile> tiles;
  std::vector<int> map;
  make_tiles(ca, cb, cc, pairs, tiles, map, ids);
  Tile* dt = nullptr; int2* dp = nullptr; int* dm = nullptr;
  TRY(dev_upload(p, tiles, &dt, s)); tmp.push_back(dt);
  TRY(dev_upload(p, pairs, &dp, s)); tmp.push_back(dp);
  TRY(dev_upload(p, map, &dm, s)); tmp.push_back(dm);
  ContractArgs c{};
  c.fields = f;
  c.nvox = slab_vox;
  c.ns = nf;
  c.tiles = dt;
  c.pairs = dp;
  c.tile_map = dm;
  c.ntiles = (int)tiles.size();
  c.gridx = pick_gridx_n(p->n_sm, c.ntiles, slab_vox);
  void* part = nullptr; void* ms = nullptr;
  TRY(dev_alloc(p, (size_t)c.gridx * c.ntiles * 16 * sizeof(double), &part)); tmp.push_back(part);
  TRY(dev_alloc(p, ca.size() * sizeof(double), &ms)); tmp.push_back(ms);
  c.partial = static_cast<double*>(part);
  c.msum = static_cast<double*>(ms);
  c.n_out = (int)ca.size();
  c.scale = 1.0;  // scaled to the ng^3 grid on the host
  for (int k = 0; k < nsl; ++k) {
    if (slab) {  // the slab's fields, [nf][x - x0][y][z]
      const int x0 = k * nx, len = std::min(nx, S - x0);
      const int nzk = zoff[k + 1] - zoff[k];
      c.nvox = (long long)len * S * S;
      TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2, f, dxi, 0, dyi, 0, dzi + zoff[k], nzk, lxy, lz, s, 0, false,
                             true, x0, len));
      if (lengths)
        TRY(run_passes<double>(p, nullptr, 0, tw, g1, g2w, static_cast<double*>(f) + (size_t)p->ns * c.nvox, dxi, 0,
                               dyi, 0, dzi + zoff[k], nzk, lxy, lz, s, 1, false, true, x0, len));
    }
    c.accumulate = k > 0;
    TRY(launch_contract_simt<double>(c, s));
    TRY(launch_reduce_partials(c, s));
  }
  tsum.assign(ca.size(), 0.0);
  cudaError_t e = cudaMemcpyAsync(tsum.data(), ms, ca.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cleanup(); return cuda_fail(e, "triangle counts"); }
  cleanup();
#undef TRY
  return BSP_OK;
}

// The contraction of a plan (CUDA cores or tensor cores) and its cross-block sums into msum.
// `mid` (optional) is recorded between the two launches. Tensor-core plans read the split fields
// of the plan's own buffer (their tensor maps point there): `fields` must be p->fields.
template <typename T>
bsp_status run_contract(bsp_plan* p, const void* fields, double* msum, cudaStream_t s, cudaEvent_t mid,
                        bool levels_ready = false) {
  bsp_status st;
  // contraction kernels of every level (lower levels first sample their fields)
  for (ContractLevel& L : p->levels) {
    const void* f = fields;
    if (!L.top && levels_ready) {
      f = L.fields;  // written by the split Z pass
    } else if (!L.top) {
      if (p->prec == BSP_MIXED_BF16X3)  // split planes sampled as 2 x shells bf16 fields
        st = launch_decimate<uint16_t>(fields, p->ngs, L.d_shells, 2 * (int)L.shells.size(), L.fields, L.g, L.stride,
                                       p->n_sm, s);
      else
        st = launch_decimate<T>(fields, p->ngs, L.d_shells, (int)L.shells.size(), L.fields, L.g, L.stride, p->n_sm, s);
      if (st != BSP_OK) return st;
      f = L.fields;
    }
    if (p->prec == BSP_MIXED_BF16X3) {
      TcArgs a{};
      a.nvox = L.nvox();
      a.ns = (int)L.shells.size();
      a.np = L.np;
      a.pair_ab = L.d_tc_pairs;
      a.n_mtiles = L.mtiles;
      a.gridy = L.gridy;
      a.vox_per_block = L.vpb;
      a.partial = L.tc_partial;
      a.error = p->d_error;
      st = launch_contract_tc(a, &L.tmap, s);
    } else {
      ContractArgs c{};
      c.fields = f;
      c.nvox = L.nvox();
      c.ns = (int)L.shells.size();
      c.tiles = L.d_tiles;
      c.pairs = L.d_pairs;
      c.tile_map = L.d_map;
      c.ntiles = L.ntiles;
      c.gridx = L.gridx;
      c.partial = L.partial;
      c.msum = msum;
      c.n_out = (int)L.bins.size();
      c.scale = L.scale;
      st = launch_contract_simt<T>(c, s);
    }
    if (st != BSP_OK) return st;
  }
  if (mid) BSP_CUDA(cudaEventRecord(mid, s));
  // cross-block sums of every level, scaled to the ng^3 grid
  if (p->prec == BSP_MIXED_BF16X3) return launch_reduce_tc_all(p->d_tc_bins, (int)p->trips.size(), msum, s);
  for (ContractLevel& L : p->levels) {
    {
      ContractArgs c{};
      c.tile_map = L.d_map;
      c.ntiles = L.ntiles;
      c.gridx = L.gridx;
      c.partial = L.partial;
      c.msum = msum;
      c.scale = L.scale;
      st = launch_reduce_partials(c, s);
    }
    if (st != BSP_OK) return st;
  }
  return BSP_OK;
}

// Kernels launched by run_contract.
int contract_launches(const bsp_plan* p) {
  int n = 0;
  for (const ContractLevel& L : p->levels) {
    const bool work = p->prec == BSP_MIXED_BF16X3 ? L.mtiles > 0 : L.ntiles > 0;
    const bool sampled = !L.top && !(p->prec == BSP_MIXED_BF16X3 && p->n_zlev > 0);  // else the Z pass did it
    n += sampled + (p->prec == BSP_MIXED_BF16X3 ? 1 : 2) * work;
  }
  return n + (p->prec == BSP_MIXED_BF16X3 ? 1 : 0);  // one cross-block sum for all tensor-core levels
}

// The contraction of x-slab k of an x-slab plan (one level, the evaluation grid) on the slab's
// fields in p->fields, its sums added to msum after the first slab.
template <typename T>
bsp_status contract_slab(bsp_plan* p, int k, cudaStream_t s) {
  if (p->levels.empty() || p->levels[0].ntiles == 0) return BSP_OK;
  const ContractLevel& L = p->levels[0];
  ContractArgs c{};
  c.fields = p->fields;
  c.nvox = (long long)p->slab_len(k) * p->ngs * p->ngs;
  c.ns = p->ns;
  c.tiles = L.d_tiles;
  c.pairs = L.d_pairs;
  c.tile_map = L.d_map;
  c.ntiles = L.ntiles;
  c.gridx = L.gridx;
  c.partial = L.partial;
  c.msum = p->msum;
  c.n_out = (int)L.bins.size();
  c.scale = L.scale;
  c.accumulate = k > 0;
  bsp_status st = launch_contract_simt<T>(c, s);
  if (st != BSP_OK) return st;
  return launch_reduce_partials(c, s);
}

// The pass launches of an estimate on the plan's buffers; ev (optional) receives an event after
// the X and after the Y pass, and after the Z pass. split: write split fields (the layout of the
// tensor-core contraction, see TcArgs) instead of FP32 ones.
template <typename T>
bsp_status plan_passes(bsp_plan* p, const void* spec, void* fields, cudaStream_t s, cudaEvent_t* ev, bool split,
                       int part) {
  PassArgs a{};
  a.n_sm = p->n_sm;
  a.spec = spec;
  a.g1 = p->g1;
  a.g2 = p->g2;
  a.fields = fields;
  a.tw = p->tw;
  a.geom = p->d_geom;
  a.ng = p->ng;
  a.ngs = p->ngs;
  a.rsd = p->rsd;
  a.beta = p->beta;
  a.rmax = p->rmax;
  a.stw = p->d_stw;
  a.stw_half = p->d_stw_half;
  bsp_status st;
  if (std::is_same<T, float>::value && p->warp_fft) {
    a.split_lo = split ? (long long)p->ns * p->nvox() / 2 : 0;
    if (split) {
      a.zlev = p->d_zlev;
      a.zmask = p->d_zmask;
      a.n_zlev = p->n_zlev;
    }
    if (part < 0) {
      a.items = p->d_wxi;
      st = launch_warp_xpass(a, p->nwxi, s);
      if (st != BSP_OK) return st;
      if (ev) BSP_CUDA(cudaEventRecord(ev[0], s));
      a.items = p->d_wyi;
      a.grid_blocks = p->y_blocks;
      st = launch_warp_ypass(a, p->nwyi, s);
      if (st != BSP_OK) return st;
      if (ev) BSP_CUDA(cudaEventRecord(ev[1], s));
      if (part == kPassXY) return BSP_OK;
    }
    a.grid_blocks = p->z_blocks;
    long long lines = (long long)p->ns * p->ngs * p->ngs;
    if (part >= 0) {
      a.slab_x0 = p->slab_x0(part);
      a.slab_nx = p->slab_len(part);
      lines = (long long)p->ns * a.slab_nx * p->ngs;
    }
    st = launch_warp_zpass(a, lines, p->n_sm, s);
    if (st != BSP_OK) return st;
    if (ev && part == kPassAll) BSP_CUDA(cudaEventRecord(ev[2], s));
    return BSP_OK;
  }
  if (p->dim == 2) {  // 2D rings: X pass, then the C2R along y on its rows (the Y stage is empty)
    a.st = p->st_full;
    a.items = p->d_xi;
    if ((st = launch_ring_xpass<T>(a, p->nxi, p->lines_xy, s)) != BSP_OK) return st;
    if (ev) {
      BSP_CUDA(cudaEventRecord(ev[0], s));
      BSP_CUDA(cudaEventRecord(ev[1], s));
    }
    a.items = p->d_zi;
    a.st = p->st_half;
    a.g2 = p->g1;
    a.slab_x0 = 0;
    a.slab_nx = 1;
    if ((st = launch_zpass<T>(a, p->nzi, p->lines_z, s)) != BSP_OK) return st;
    if (ev) BSP_CUDA(cudaEventRecord(ev[2], s));
    return BSP_OK;
  }
  if (part < 0) {
    a.st = p->st_full;
    a.items = p->d_xi;
    st = launch_xpass<T>(a, p->nxi, p->lines_xy, s);
    if (st != BSP_OK) return st;
    if (ev) BSP_CUDA(cudaEventRecord(ev[0], s));
    a.items = p->d_yi;
    st = launch_ypass<T>(a, p->nyi, p->lines_xy, s);
    if (st != BSP_OK) return st;
    if (ev) BSP_CUDA(cudaEventRecord(ev[1], s));
    if (part == kPassXY) return BSP_OK;
  }
  a.items = p->d_zi;
  int nzi = p->nzi;
  if (part >= 0) {
    a.items = p->d_zi + p->zi_off[part];
    nzi = p->zi_off[part + 1] - p->zi_off[part];
    a.slab_x0 = p->slab_x0(part);
    a.slab_nx = p->slab_len(part);
  }
  a.st = p->st_half;
  if (split) a.fields = p->fields32;
  st = launch_zpass<T>(a, nzi, p->lines_z, s);
  if (st != BSP_OK) return st;
  if (split) {
    st = launch_split_fields(static_cast<const float*>(p->fields32), static_cast<uint32_t*>(fields),
                             (long long)p->ns * p->nvox() / 2, p->n_sm, s);
    if (st != BSP_OK) return st;
  }
  if (ev && part == kPassAll) BSP_CUDA(cudaEventRecord(ev[2], s));
  return BSP_OK;
}

template <typename T>
bsp_status estimate_impl(bsp_plan* p, const void* spec, double* b_trip, double* b_grid, cudaStream_t s) {
  const bool rec = p->timing_on && p->timing_calls < p->timing_max;
  cudaEvent_t* ev = rec ? &p->events[(size_t)p->timing_calls * (BSP_N_STAGES + 1)] : nullptr;
  if (rec) BSP_CUDA(cudaEventRecord(ev[0], s));
  const bool split = p->prec == BSP_MIXED_BF16X3;
  bsp_status st;
  if (p->slab_nx) {
    // memory budget: X and Y passes once, then the Z pass and the contraction slab by slab (the
    // timing's Z-pass stage covers all slabs' Z passes and contractions)
    st = plan_passes<T>(p, spec, p->fields, s, rec ? ev + 1 : nullptr, false, kPassXY);
    if (st != BSP_OK) return st;
    for (int k = 0; k < p->n_slabs(); ++k) {
      if ((st = plan_passes<T>(p, spec, p->fields, s, nullptr, false, k)) != BSP_OK) return st;
      if ((st = contract_slab<T>(p, k, s)) != BSP_OK) return st;
    }
    if (rec) {
      BSP_CUDA(cudaEventRecord(ev[3], s));
      BSP_CUDA(cudaEventRecord(ev[4], s));
    }
  } else {
    st = plan_passes<T>(p, spec, p->fields, s, rec ? ev + 1 : nullptr, split);
    if (st != BSP_OK) return st;
    if (p->order == 4) {  // product fields d_c d_e after the shell fields
      st = launch_pair_fields<T>(p->fields, p->nvox(), p->d_pairs4, p->n_extra(),
                                 static_cast<T*>(p->fields) + (size_t)p->ns * p->nvox(), p->n_sm, s);
      if (st != BSP_OK) return st;
    }
    st = run_contract<T>(p, p->fields, p->msum, s, rec ? ev[4] : nullptr, split && p->warp_fft);
    if (st != BSP_OK) return st;
  }
  FinalizeArgs f{};
  f.msum = p->msum;
  f.tsum = p->tsum;
  f.n_trip = (int)p->trips.size();
  f.cell_ptr = p->cell_ptr;
  f.cell_idx = p->cell_idx;
  f.n_cells = p->n_cells();
  const double vc = pow(p->box_len / p->ng, (double)p->dim);  // cell volume (area in 2D)
  f.norm = pow(vc, (double)p->order) / pow(p->box_len, (double)p->dim);
  f.b_trip = b_trip;
  f.b_grid = b_grid;
  st = launch_finalize(f, s);
  if (st != BSP_OK) return st;
  if (rec) {
    BSP_CUDA(cudaEventRecord(ev[5], s));
    p->timing_calls += 1;
    if (p->slab_nx) {
      int passes = p->warp_fft ? 2 + p->n_slabs() : (p->nxi > 0) + (p->nyi > 0);
      if (!p->warp_fft)
        for (int k = 0; k < p->n_slabs(); ++k) passes += p->zi_off[k + 1] > p->zi_off[k];
      const bool work = !p->levels.empty() && p->levels[0].ntiles > 0;
      p->launches += passes + 2LL * work * p->n_slabs() + 1;
    } else {
      const int passes = (p->warp_fft ? 3 : (p->nxi > 0) + (p->nyi > 0) + (p->nzi > 0) + (split ? 1 : 0)) +
                         (p->order == 4);
      p->launches += passes + contract_launches(p) + 1;
    }
  }
  return BSP_OK;
}

// Algorithmic bytes and flops of each stage of one estimate (see bsp_plan_stage_work).
void stage_work(const bsp_plan* p, double* bytes, double* flops) {
  const double ce = 2.0 * p->elem();
  const double re = (double)p->elem();
  const double ng = (double)p->ngs;
  for (int i = 0; i < BSP_N_STAGES; ++i) { bytes[i] = 0.0; flops[i] = 0.0; }
  for (int n = 0; n < p->ns && p->dim == 2; ++n) {  // 2D: X pass over k_y < r lines, C2R along y
    const ShellGeom& g = p->geom[n];
    long long modes_half = 0;
    for (int ky = 0; ky < g.r; ++ky)
      for (int kx = -(g.r - 1); kx <= g.r - 1; ++kx) {
        const long long q = (long long)kx * kx + (long long)ky * ky;
        if (q >= g.qlo && q < g.qhi) modes_half += 1;
      }
    bytes[BSP_STAGE_XPASS] += ce * (double)modes_half + ce * ng * g.r;
    bytes[BSP_STAGE_ZPASS] += ce * ng * g.r + re * ng * ng;
  }
  for (int n = 0; n < p->ns && p->dim == 3; ++n) {
    const ShellGeom& g = p->geom[n];
    const int r = g.r;
    long long modes_half = 0, xlines = 0;
    for (int ky = -(r - 1); ky <= r - 1; ++ky)
      for (int kz = 0; kz < r; ++kz) {
        const long long q2 = (long long)ky * ky + (long long)kz * kz;
        if (q2 >= g.qhi) continue;
        xlines += 1;
        for (int kx = -(r - 1); kx <= r - 1; ++kx) {
          const long long q = q2 + (long long)kx * kx;
          if (q >= g.qlo && q < g.qhi) modes_half += 1;
        }
      }
    bytes[BSP_STAGE_XPASS] += ce * (double)modes_half + ce * ng * (double)xlines;
    bytes[BSP_STAGE_YPASS] += ce * ng * (double)xlines + ce * ng * ng * r;
    bytes[BSP_STAGE_ZPASS] += ce * ng * ng * r + re * ng * ng * ng;
  }
  // contraction levels: fields read once per level (lower levels also read their samples of the
  // evaluation grid and write them), work per level on its g^3 grid
  for (const ContractLevel& L : p->levels) {
    const double nv = (double)L.nvox();
    const double nsh = (double)L.shells.size();
    long long npairs = 0;
    for (size_t i = 0; i < L.bins.size(); ++i) {
      const bsp_triplet& a = p->trips[L.bins[i]];
      if (i == 0 || a.a != p->trips[L.bins[i - 1]].a || a.b != p->trips[L.bins[i - 1]].b) npairs += 1;
    }
    bytes[BSP_STAGE_CONTRACT] += re * nsh * nv * (L.top ? 1.0 : 3.0);
    if (p->prec == BSP_MIXED_BF16X3)
      flops[BSP_STAGE_CONTRACT] += 3.0 * 2.0 * (double)npairs * (double)L.np * nv;  // split-BF16 GEMM
    else
      flops[BSP_STAGE_CONTRACT] += ((double)npairs + 2.0 * (double)L.bins.size()) * nv;
  }
  bytes[BSP_STAGE_FINALIZE] = 8.0 * (double)p->trips.size() * 3 + 8.0 * p->n_cells();
}


// Resources of the ng-grid transforms over the union of the shells (the ball of every shell
// mode): twiddles, one pseudo-shell geometry, work items, pass buffers.
bsp_status ball_setup(bsp_plan* p, cudaStream_t s) {
  if (p->ball_ready) return BSP_OK;
  bsp_status st;
  if ((st = dev_alloc(p, (size_t)p->ng * sizeof(float2), &p->d_tw_ng)) != BSP_OK) return st;
  if ((st = launch_twiddles<float>(p->d_tw_ng, p->ng, s)) != BSP_OK) return st;
  {
    std::vector<float2> t1, t2;
    warp_stage_table(p->ng, t1);
    warp_stage_table(p->ng / 2, t2);
    if (t1.empty()) t1.assign(1, make_float2(0.f, 0.f));
    if (t2.empty()) t2.assign(1, make_float2(0.f, 0.f));
    if ((st = dev_upload(p, t1, &p->d_stw_ng, s)) != BSP_OK) return st;
    if ((st = dev_upload(p, t2, &p->d_stw_ng_half, s)) != BSP_OK) return st;
  }
  // the final inverse transform covers the union of the shells as one pseudo-shell
  std::vector<ShellGeom> ball(1);
  ball[0].qlo = (int)p->q[0];
  ball[0].qhi = (int)p->q[p->ns];
  ball[0].r = (int)isqrt_ll(p->q[p->ns] - 1) + 1;
  ball[0].pad = 0;
  ball[0].g1_off = 0;
  ball[0].g2_off = 0;
  std::vector<Item> bx, by, bz;
  make_items_g(ball, p->ng, warp_fft_lines(), 1, bx, by, bz);
  p->nbxi = (int)bx.size();
  p->nbyi = (int)by.size();
  if ((st = dev_upload(p, ball, &p->d_ball, s)) != BSP_OK) return st;
  if ((st = dev_upload(p, bx, &p->d_bxi, s)) != BSP_OK) return st;
  if ((st = dev_upload(p, by, &p->d_byi, s)) != BSP_OK) return st;
  const long long r = ball[0].r;
  if ((st = dev_alloc(p, (size_t)p->ng * (2 * r - 1) * r * sizeof(float2), &p->g1b)) != BSP_OK) return st;
  if ((st = dev_alloc(p, (size_t)p->ng * p->ng * r * sizeof(float2), &p->g2b)) != BSP_OK) return st;
  p->ball_ready = true;
  return BSP_OK;
}

// Resources of the gradient: adjoint pair table, W entries, buffers (first bsp_grad call).
bsp_status grad_setup(bsp_plan* p, cudaStream_t s) {
  if (p->grad_ready) return BSP_OK;
  const int ns = p->ns;
  p->adj_np = ns <= 32 ? 32 : 64;
  const int np = p->adj_np;
  // every unordered pair (x >= y) that is the complement of a bin position
  std::vector<int> pid((size_t)ns * ns, -1);
  std::vector<int2> pairs;
  auto pair_index = [&](int x, int y) {
    if (x < y) std::swap(x, y);
    int& e = pid[(size_t)x * ns + y];
    if (e < 0) { e = (int)pairs.size(); pairs.push_back(make_int2(x, y)); }
    return e;
  };
  std::vector<std::vector<int>> lists;
  auto add = [&](int pr, int n, int t) {
    const size_t e = (size_t)pr * np + n;
    if (lists.size() <= e) lists.resize(e + 1);
    lists[e].push_back(t);
  };
  for (size_t t = 0; t < p->trips.size(); ++t) {
    const bsp_triplet& b = p->trips[t];
    add(pair_index(b.b, b.c), b.a, (int)t);
    add(pair_index(b.a, b.c), b.b, (int)t);
    add(pair_index(b.a, b.b), b.c, (int)t);
  }
  p->adj_npairs = (int)pairs.size();
  p->adj_entries = p->adj_npairs * np;
  lists.resize(p->adj_entries);
  std::vector<int> ptr(p->adj_entries + 1, 0), idx;
  for (int e = 0; e < p->adj_entries; ++e) {
    ptr[e + 1] = ptr[e] + (int)lists[e].size();
    idx.insert(idx.end(), lists[e].begin(), lists[e].end());
  }
  const double vc = pow(p->box_len / p->ng, 3.0);
  const double norm = vc * vc * vc / (p->box_len * p->box_len * p->box_len);
  std::vector<double> cnorm(p->trips.size());
  for (size_t t = 0; t < p->trips.size(); ++t) cnorm[t] = norm / p->trips[t].tsum;
  bsp_status st;
  void* tmp = nullptr;
  if ((st = dev_upload(p, pairs, &p->d_adj_pairs, s)) != BSP_OK) return st;
  if ((st = dev_upload(p, ptr, &p->d_w_ptr, s)) != BSP_OK) return st;
  if ((st = dev_upload(p, idx, &p->d_w_idx, s)) != BSP_OK) return st;
  if ((st = dev_upload(p, cnorm, &p->d_cnorm, s)) != BSP_OK) return st;
  if ((st = dev_alloc(p, (size_t)p->adj_entries * sizeof(float), &tmp)) != BSP_OK) return st;
  p->d_w = static_cast<float*>(tmp);
  if ((st = dev_alloc(p, p->store_bytes(), &tmp)) != BSP_OK) return st;  // G_n of the grid or of one x-slab
  p->d_gfields = static_cast<float*>(tmp);
  if ((st = dev_alloc(p, (size_t)p->ng * p->ng * (p->ng / 2 + 1) * sizeof(float2), &p->d_grad_spec)) != BSP_OK)
    return st;
  if ((st = ball_setup(p, s)) != BSP_OK) return st;
  p->grad_ready = true;
  return BSP_OK;
}
}  // namespace

extern "C" {

const char* bsp_last_error(void) { return g_error; }

const char* bsp_version(void) { return "bispec-gb300 0.1 (sm_103a)"; }

bsp_status bsp_plan_create(const bsp_plan_desc* desc, void* stream, bsp_plan** out) {
  if (!out) return fail(BSP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  g_error[0] = 0;
  bsp_status st = validate(desc);
  if (st != BSP_OK) return st;
  bsp_plan* p = new (std::nothrow) bsp_plan();
  if (!p) return fail(BSP_ERR_OOM, "host allocation failed");
  st = host_plan(p, desc);
  if (st != BSP_OK) { delete p; return st; }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "device query"); }
  // candidate bins: the triangle inequality on the extreme mode lengths (order 4: the largest
  // side of a closed quadrilateral is at most the sum of the others); an order-4 bin (a, b, c, e)
  // is summed as the triple (a, b, ns + pid4(c, e)) of shell fields and pair-product fields
  std::vector<int> ca, cb, cc, c4;
  auto qmaxr = [&](int n) { return sqrt((double)(p->q[n + 1] - 1)); };
  for (int a = 0; a < p->ns; ++a)
    for (int b = 0; b <= a; ++b)
      for (int c = 0; c <= b; ++c) {
        const double ra = sqrt((double)p->q[a]);
        if (p->order == 3) {
          if (ra <= qmaxr(b) + qmaxr(c)) { ca.push_back(a); cb.push_back(b); cc.push_back(c); c4.push_back(-1); }
          continue;
        }
        for (int e = 0; e <= c; ++e)
          if (ra <= qmaxr(b) + qmaxr(c) + qmaxr(e)) {
            ca.push_back(a); cb.push_back(b); cc.push_back(c); c4.push_back(e);
          }
      }
  // geometry on the device (shared by the FP64 count and the estimator)
  st = dev_upload(p, p->geom, &p->d_geom, s);
  if (st != BSP_OK) { bsp_plan_destroy(p); return st; }
  std::vector<int> cc_sum = cc;  // the third index of each candidate's triple sum
  if (p->order == 4) {
    for (int c = 0; c < p->ns; ++c)
      for (int e = 0; e <= c; ++e) p->pairs4.push_back(make_int2(c, e));
    st = dev_upload(p, p->pairs4, &p->d_pairs4, s);
    if (st != BSP_OK) { bsp_plan_destroy(p); return st; }
    for (size_t i = 0; i < cc.size(); ++i) cc_sum[i] = p->ns + p->pid4(cc[i], c4[i]);
  }
  std::vector<double> tsum;
  st = plan_sums(p, false, ca, cb, cc_sum, nullptr, tsum, s);
  if (st != BSP_OK) { bsp_plan_destroy(p); return st; }
  for (double& t : tsum) t *= p->sum_scale;  // sums over the ng^3 grid (exact up to rounding)
  const double ng3 = p->dim == 2 ? (double)p->ng * (double)p->ng : (double)p->ng * (double)p->ng * (double)p->ng;
  std::vector<int> ka, kb, kc;
  std::vector<double> kt;
  for (size_t i = 0; i < ca.size(); ++i) {
    const double nt = tsum[i] / ng3;
    const double rn = rint(nt);
    if (fabs(nt - rn) > 1e-3) {
      bsp_plan_destroy(p);
      return fail(BSP_ERR_NUMERIC, "non-integral triangle count for bin (" + std::to_string(ca[i]) + "," +
                                       std::to_string(cb[i]) + "," + std::to_string(cc[i]) +
                                       (c4[i] >= 0 ? "," + std::to_string(c4[i]) : std::string()) + ")");
    }
    if (rn <= 0.0) continue;
    ka.push_back(ca[i]); kb.push_back(cb[i]); kc.push_back(cc[i]);
    kt.push_back(tsum[i]);
    bsp_triplet t{};
    t.a = ca[i]; t.b = cb[i]; t.c = cc[i]; t.e = c4[i];
    t.ntri = rn;
    t.tsum = tsum[i];
    t.k1 = p->kbar[t.a]; t.k2 = p->kbar[t.b]; t.k3 = p->kbar[t.c];
    p->trips.push_back(t);
  }
  if (p->label_k == BSP_LABEL_TRIANGLE_MEAN && !p->trips.empty()) {
    // mean side lengths over each bin's triangles: sum w_a i_b i_c / sum i_a i_b i_c and the
    // other two placements of w, with the count itself in the same launch (4 sums per bin)
    struct E { int a, b, c, id; };
    std::vector<E> ent;
    const int ns = p->ns;
    for (size_t i = 0; i < p->trips.size(); ++i) {
      const bsp_triplet& t = p->trips[i];
      const int id = 4 * (int)i;
      ent.push_back({ns + t.a, t.b, t.c, id});
      ent.push_back({t.a, ns + t.b, t.c, id + 1});
      ent.push_back({t.a, t.b, ns + t.c, id + 2});
      ent.push_back({t.a, t.b, t.c, id + 3});
    }
    std::sort(ent.begin(), ent.end(), [](const E& x, const E& y) {
      return x.a != y.a ? x.a < y.a : x.b != y.b ? x.b < y.b : x.c < y.c;
    });
    std::vector<int> ea, eb, ec, eid;
    for (const E& x : ent) { ea.push_back(x.a); eb.push_back(x.b); ec.push_back(x.c); eid.push_back(x.id); }
    std::vector<double> ks;
    st = plan_sums(p, true, ea, eb, ec, &eid, ks, s);
    if (st != BSP_OK) { bsp_plan_destroy(p); return st; }
    for (size_t i = 0; i < p->trips.size(); ++i) {
      bsp_triplet& t = p->trips[i];
      const double tt = ks[4 * i + 3];
      t.k1 = ks[4 * i] / tt; t.k2 = ks[4 * i + 1] / tt; t.k3 = ks[4 * i + 2] / tt;
    }
  }
  for (bsp_triplet& t : p->trips) {  // Eq. (2.4) and the (mu, t) cell
    if (p->order == 4) {  // no triangle shape: every bin in the one cell of its k1 group
      t.mu = t.t = NAN;
      t.i_mu = t.i_t = t.inside = 0;
      continue;
    }
    const double k1 = t.k1, k2 = t.k2, k3 = t.k3;
    t.t = k2 / k1;
    t.mu = 0.5 * (k1 / k2 + k2 / k1 - (k3 / k1) * (k3 / k2));
    const double mc = std::min(std::max(t.mu, 0.5), 1.0);
    const double tc = std::min(std::max(t.t, 0.5), 1.0);
    t.i_mu = std::min((int)floor((mc - 0.5) * (2.0 * p->n_mu)), p->n_mu - 1);
    t.i_t = std::min((int)floor((tc - 0.5) * (2.0 * p->n_t)), p->n_t - 1);
    t.inside = (t.t >= 0.5 && t.t <= 1.0 && t.mu >= 0.5 && t.mu <= 1.0 && 2.0 * t.mu * t.t >= 1.0) ? 1 : 0;
  }
  // estimator buffers in the plan's precision
  p->lines_xy = fft_lines_for(p->ngs, p->prec);
  p->lines_z = fft_lines_for(p->ngs / 2, p->prec);
  std::vector<Item> xi, yi, zi;
  make_items(p, p->lines_xy, p->lines_z, xi, yi, zi);
  p->nxi = (int)xi.size(); p->nyi = (int)yi.size(); p->nzi = (int)zi.size();
  const size_t ce = p->prec == BSP_FP64 ? sizeof(double2) : sizeof(float2);
  std::vector<int> cptr(p->n_cells() + 1, 0), cidx;
  {
    std::vector<std::vector<int>> cells(p->n_cells());
    for (size_t t = 0; t < p->trips.size(); ++t) {
      const bsp_triplet& b = p->trips[t];
      cells[((b.a / p->k1_merge) * p->n_mu + b.i_mu) * p->n_t + b.i_t].push_back((int)t);
    }
    for (int c = 0; c < p->n_cells(); ++c) {
      cptr[c + 1] = cptr[c] + (int)cells[c].size();
      cidx.insert(cidx.end(), cells[c].begin(), cells[c].end());
    }
  }
#define TRY(x) do { st = (x); if (st != BSP_OK) { bsp_plan_destroy(p); return st; } } while (0)
  TRY(dev_alloc(p, p->ngs * ce, &p->tw));
  TRY(p->prec == BSP_FP64 ? launch_twiddles<double>(p->tw, p->ngs, s) : launch_twiddles<float>(p->tw, p->ngs, s));
  TRY(dev_upload(p, xi, &p->d_xi, s));
  TRY(dev_upload(p, yi, &p->d_yi, s));
  slab_items(p->slab_nx, p->ngs, zi, p->zi_off);
  TRY(dev_upload(p, zi, &p->d_zi, s));
  for (const ShellGeom& g : p->geom) p->rmax = std::max(p->rmax, g.r);
  p->warp_fft = p->dim == 3 && p->prec != BSP_FP64 && warp_fft_supported(p->ngs);
  if (p->warp_fft) {
    std::vector<float2> t1, t2;
    warp_stage_table(p->ngs, t1);
    warp_stage_table(p->ngs / 2, t2);
    if (t2.empty()) t2.assign(1, make_float2(0.f, 0.f));
    TRY(dev_upload(p, t1, &p->d_stw, s));
    TRY(dev_upload(p, t2, &p->d_stw_half, s));
    std::vector<Item> wx, wy, wz;
    make_items(p, warp_fft_lines(), 1, wx, wy, wz);
    p->nwxi = (int)wx.size();
    p->nwyi = (int)wy.size();
    TRY(dev_upload(p, wx, &p->d_wxi, s));
    TRY(dev_upload(p, wy, &p->d_wyi, s));
  }
  TRY(dev_alloc(p, g1_elems(p) * ce, &p->g1));
  TRY(dev_alloc(p, g2_elems(p) * ce, &p->g2));
  TRY(dev_alloc(p, p->store_bytes(), &p->fields));  // all fields, or one x-slab of them
  if (p->prec == BSP_MIXED_BF16X3 && !p->warp_fft) TRY(dev_alloc(p, p->field_bytes(), &p->fields32));
  TRY(build_levels(p, s));
  if (p->autotune) TRY(autotune_passes(p, s));
  void* tmp = nullptr;
  TRY(dev_alloc(p, std::max<size_t>(p->trips.size(), 1) * sizeof(double), &tmp));
  p->msum = static_cast<double*>(tmp);
  TRY(dev_upload(p, kt, &p->tsum, s));
  {
    std::vector<int> zero(1, 0);
    TRY(dev_upload(p, zero, &p->d_error, s));
  }
  TRY(dev_upload(p, cptr, &p->cell_ptr, s));
  TRY(dev_upload(p, cidx, &p->cell_idx, s));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { bsp_plan_destroy(p); return cuda_fail(e, "plan upload"); }
#undef TRY
  *out = p;
  return BSP_OK;
}

bsp_status bsp_plan_destroy(bsp_plan* p) {
  if (!p) return BSP_OK;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  p->events.clear();
  for (auto& b : p->bufs) cudaFree(b.p);
  p->bufs.clear();
  delete p;
  return BSP_OK;
}

bsp_status bsp_plan_info(const bsp_plan* p, int* n_triplets, int* n_shells, size_t* field_bytes,
                         size_t* device_bytes) {
  if (!p) return fail(BSP_ERR_INVALID_ARG, "plan is NULL");
  if (n_triplets) *n_triplets = (int)p->trips.size();
  if (n_shells) *n_shells = p->ns;
  if (field_bytes) *field_bytes = p->field_bytes();
  if (device_bytes) *device_bytes = p->dev_bytes;
  return BSP_OK;
}

bsp_status bsp_plan_tuning(const bsp_plan* p, int* n_levels, int* level_side, int* blocks_mult, int max_levels) {
  if (!p || !n_levels) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *n_levels = (int)p->levels.size();
  for (int l = 0; l < (int)p->levels.size() && l < max_levels; ++l) {
    if (level_side) level_side[l] = p->levels[l].g;
    if (blocks_mult) blocks_mult[l] = p->prec == BSP_MIXED_BF16X3 ? p->levels[l].tune_mult : 0;
  }
  return BSP_OK;
}

bsp_status bsp_plan_grid(const bsp_plan* p, int* ng_eval) {
  if (!p || !ng_eval) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *ng_eval = p->ngs;
  return BSP_OK;
}

bsp_status bsp_plan_triplets(const bsp_plan* p, const bsp_triplet** table, int* n) {
  if (!p || !table || !n) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *table = p->trips.data();
  *n = (int)p->trips.size();
  return BSP_OK;
}

bsp_status bsp_shell_fields(bsp_plan* p, const void* spec, void* fields_out, void* stream) {
  if (!p || !spec || !fields_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->prec == BSP_FP64) return plan_passes<double>(p, spec, fields_out, s, nullptr);
  return plan_passes<float>(p, spec, fields_out, s, nullptr);
}

bsp_status bsp_contract(bsp_plan* p, const void* fields, double* msum, void* stream) {
  if (!p || !fields || !msum) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if ((reinterpret_cast<uintptr_t>(fields) & 15) != 0) return fail(BSP_ERR_INVALID_ARG, "fields must be 16-byte aligned");
  if (p->order == 4) return fail(BSP_ERR_NOT_SUPPORTED, "bsp_contract: order-4 plans sum pair-product fields");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->prec == BSP_FP64) return run_contract<double>(p, fields, msum, s, nullptr);
  if (p->prec == BSP_MIXED_BF16X3) {
    // the tensor-core contraction reads split fields from the plan's buffer
    const bsp_status st = launch_split_fields(static_cast<const float*>(fields), static_cast<uint32_t*>(p->fields),
                                              (long long)p->ns * p->nvox() / 2, p->n_sm, s);
    if (st != BSP_OK) return st;
    return run_contract<float>(p, p->fields, msum, s, nullptr);
  }
  return run_contract<float>(p, fields, msum, s, nullptr);
}

bsp_status bsp_plan_check(bsp_plan* p, void* stream) {
  if (!p) return fail(BSP_ERR_INVALID_ARG, "plan is NULL");
  BSP_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int flag = 0;
  BSP_CUDA(cudaMemcpy(&flag, p->d_error, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) return fail(BSP_ERR_TIMEOUT, "a bounded device-side wait gave up in an earlier call");
  return BSP_OK;
}

bsp_status bsp_estimate(bsp_plan* p, const void* spec, double* b_triplet, double* b_grid, void* stream) {
  if (!p || !spec || !b_triplet) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->prec == BSP_FP64) return estimate_impl<double>(p, spec, b_triplet, b_grid, s);
  return estimate_impl<float>(p, spec, b_triplet, b_grid, s);
}

bsp_status bsp_estimate_batched(bsp_plan* const* plans, const void* const* specs, int n, double* const* b_triplet,
                                double* const* b_grid, void* stream) {
  if (n < 0 || (n > 0 && (!plans || !specs || !b_triplet))) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < n; ++i) {
    bsp_status st = bsp_estimate(plans[i], specs[i], b_triplet[i], b_grid ? b_grid[i] : nullptr, stream);
    if (st != BSP_OK) return st;
  }
  return BSP_OK;
}

bsp_status bsp_batch_create(bsp_plan* const* plans, const void* const* specs, int n, double* const* b_triplet,
                            double* const* b_grid, void* stream, bsp_batch** out) {
  if (!out) return fail(BSP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || !plans || !specs || !b_triplet) return fail(BSP_ERR_INVALID_ARG, "NULL argument or n < 1");
  for (int i = 0; i < n; ++i) {
    if (!plans[i] || !specs[i] || !b_triplet[i]) return fail(BSP_ERR_INVALID_ARG, "NULL entry");
    if (plans[i]->timing_on) return fail(BSP_ERR_INVALID_ARG, "disable plan timing before capturing a batch");
  }
  // warm every distinct plan once outside capture (kernel attributes, lazy module loading)
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) {
    bool seen = false;
    for (int j = 0; j < i; ++j) seen = seen || plans[j] == plans[i];
    if (seen) continue;
    bsp_status st = bsp_estimate(plans[i], specs[i], b_triplet[i], b_grid ? b_grid[i] : nullptr, stream);
    if (st != BSP_OK) return st;
  }
  BSP_CUDA(cudaStreamSynchronize(s));
  cudaStream_t cap;
  BSP_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) { cudaStreamDestroy(cap); return cuda_fail(e, "cudaStreamBeginCapture"); }
  bsp_status st = BSP_OK;
  for (int i = 0; i < n && st == BSP_OK; ++i)
    st = bsp_estimate(plans[i], specs[i], b_triplet[i], b_grid ? b_grid[i] : nullptr, cap);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cap, &graph);
  cudaStreamDestroy(cap);
  if (st != BSP_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(e, "cudaGraphInstantiate"); }
  bsp_batch* b = new (std::nothrow) bsp_batch();
  if (!b) { cudaGraphExecDestroy(exec); cudaGraphDestroy(graph); return fail(BSP_ERR_OOM, "host allocation failed"); }
  b->graph = graph;
  b->exec = exec;
  b->n = n;
  *out = b;
  return BSP_OK;
}

bsp_status bsp_batch_run(bsp_batch* b, void* stream) {
  if (!b) return fail(BSP_ERR_INVALID_ARG, "batch is NULL");
  BSP_CUDA(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
  return BSP_OK;
}

bsp_status bsp_batch_destroy(bsp_batch* b) {
  if (!b) return BSP_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
  return BSP_OK;
}

bsp_status bsp_estimate_host(bsp_plan* p, const void* spec_host, double* b_triplet_host, double* b_grid_host,
                             void* stream) {
  if (!p || !spec_host || !b_triplet_host) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bsp_status st;
  if (!p->spec_dev) {
    st = dev_alloc(p, p->spec_bytes(), &p->spec_dev);
    if (st != BSP_OK) return st;
    void* t = nullptr;
    st = dev_alloc(p, std::max<size_t>(p->trips.size(), 1) * sizeof(double), &t);
    if (st != BSP_OK) return st;
    p->btrip_dev = static_cast<double*>(t);
    st = dev_alloc(p, (size_t)p->n_cells() * sizeof(double), &t);
    if (st != BSP_OK) return st;
    p->bgrid_dev = static_cast<double*>(t);
  }
  // Only the modes the shells can reach are read by the estimator: |m_x|, |m_y| <= R - 1 and
  // 0 <= m_z <= R - 1 with R = r of the outermost shell. Copy that box (four boxes in the
  // wrapped index ranges); the rest of the device copy is never read. 2D: rows |m_x| <= R - 1,
  // their first R entries (0 <= m_y <= R - 1).
  if (p->dim == 2) {
    const int ng = p->ng, hy = ng / 2 + 1, R = p->rmax;
    const size_t ce = 2 * p->elem();
    const int lo[2] = {0, ng - (R - 1)}, len[2] = {R, R - 1};
    for (int bx = 0; bx < 2; ++bx) {
      if (len[bx] <= 0) continue;
      const size_t off = (size_t)lo[bx] * hy * ce;
      BSP_CUDA(cudaMemcpy2DAsync(static_cast<char*>(p->spec_dev) + off, (size_t)hy * ce,
                                 static_cast<const char*>(spec_host) + off, (size_t)hy * ce, (size_t)R * ce,
                                 (size_t)len[bx], cudaMemcpyHostToDevice, s));
    }
  } else {
    const int ng = p->ng, hz = ng / 2 + 1, R = p->rmax;
    const size_t ce = 2 * p->elem();
    const int lo[2] = {0, ng - (R - 1)}, len[2] = {R, R - 1};
    for (int bx = 0; bx < 2; ++bx)
      for (int by = 0; by < 2; ++by) {
        if (len[bx] <= 0 || len[by] <= 0) continue;
        cudaMemcpy3DParms m{};
        m.srcPtr = make_cudaPitchedPtr(const_cast<void*>(spec_host), (size_t)hz * ce, (size_t)hz * ce, (size_t)ng);
        m.dstPtr = make_cudaPitchedPtr(p->spec_dev, (size_t)hz * ce, (size_t)hz * ce, (size_t)ng);
        m.srcPos = make_cudaPos(0, (size_t)lo[by], (size_t)lo[bx]);
        m.dstPos = m.srcPos;
        m.extent = make_cudaExtent((size_t)R * ce, (size_t)len[by], (size_t)len[bx]);
        m.kind = cudaMemcpyHostToDevice;
        BSP_CUDA(cudaMemcpy3DAsync(&m, s));
      }
  }
  st = bsp_estimate(p, p->spec_dev, p->btrip_dev, b_grid_host ? p->bgrid_dev : nullptr, stream);
  if (st != BSP_OK) return st;
  BSP_CUDA(cudaMemcpyAsync(b_triplet_host, p->btrip_dev, p->trips.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  if (b_grid_host)
    BSP_CUDA(cudaMemcpyAsync(b_grid_host, p->bgrid_dev, (size_t)p->n_cells() * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
  BSP_CUDA(cudaStreamSynchronize(s));
  return BSP_OK;
}

bsp_status bsp_plan_pass_tuning(const bsp_plan* p, int* y_blocks, int* z_blocks) {
  if (!p || !y_blocks || !z_blocks) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *y_blocks = p->y_blocks;
  *z_blocks = p->z_blocks;
  return BSP_OK;
}

bsp_status bsp_plan_slabs(const bsp_plan* p, int* slab_planes, int* n_slabs) {
  if (!p || !slab_planes || !n_slabs) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *slab_planes = p->slab_nx;
  *n_slabs = p->n_slabs();
  return BSP_OK;
}

bsp_status bsp_plan_host_input_bytes(const bsp_plan* p, size_t* bytes) {
  if (!p || !bytes) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  const size_t R = (size_t)p->rmax;
  *bytes = (p->dim == 2 ? 1 : 2 * R - 1) * (2 * R - 1) * R * 2 * p->elem();
  return BSP_OK;
}

bsp_status bsp_timing_enable(bsp_plan* p, int enable, int max_calls) {
  if (!p || max_calls < 0) return fail(BSP_ERR_INVALID_ARG, "bad argument");
  p->timing_on = false;
  p->timing_calls = 0;
  p->launches = 0;
  if (!enable) return BSP_OK;
  const size_t need = (size_t)max_calls * (BSP_N_STAGES + 1);
  while (p->events.size() < need) {
    cudaEvent_t e;
    BSP_CUDA(cudaEventCreate(&e));
    p->events.push_back(e);
  }
  p->timing_max = max_calls;
  p->timing_on = true;
  return BSP_OK;
}

bsp_status bsp_timing_read(bsp_plan* p, double* ms, int* n_calls, long long* n_launches) {
  if (!p || !ms) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < BSP_N_STAGES; ++i) ms[i] = 0.0;
  for (int c = 0; c < p->timing_calls; ++c) {
    cudaEvent_t* ev = &p->events[(size_t)c * (BSP_N_STAGES + 1)];
    BSP_CUDA(cudaEventSynchronize(ev[BSP_N_STAGES]));
    for (int i = 0; i < BSP_N_STAGES; ++i) {
      float t = 0.f;
      BSP_CUDA(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      ms[i] += t;
    }
  }
  if (p->timing_calls > 0)
    for (int i = 0; i < BSP_N_STAGES; ++i) ms[i] /= p->timing_calls;
  if (n_calls) *n_calls = p->timing_calls;
  if (n_launches) *n_launches = p->launches;
  return BSP_OK;
}

bsp_status bsp_plan_stage_work(const bsp_plan* p, double* bytes, double* flops) {
  if (!p || !bytes || !flops) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  stage_work(p, bytes, flops);
  return BSP_OK;
}

bsp_status bsp_spectrum(bsp_plan* p, const float* delta_x, void* spec_out, void* stream) {
  if (!p || !delta_x || !spec_out) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (p->prec == BSP_FP64 || p->dim == 2) return fail(BSP_ERR_NOT_SUPPORTED, "bsp_spectrum needs a 3D FP32 or mixed plan");
  if (!warp_fft_supported(p->ng)) return fail(BSP_ERR_NOT_SUPPORTED, "bsp_spectrum needs ng = 2^p or 3 * 2^p in [128, 1024]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bsp_status st = ball_setup(p, s);
  if (st != BSP_OK) return st;
  PassArgs b{};
  b.n_sm = p->n_sm;
  b.g1 = p->g1b;
  b.g2 = p->g2b;
  b.fields = spec_out;
  b.tw = p->d_tw_ng;
  b.geom = p->d_ball;
  b.ng = p->ng;
  b.ngs = p->ng;
  b.rsd = 0;
  b.beta = 0.0;
  b.rmax = (int)isqrt_ll(p->q[p->ns] - 1) + 1;
  b.stw = p->d_stw_ng;
  b.stw_half = p->d_stw_ng_half;
  st = launch_warp_zfpass(b, delta_x, (long long)p->ng * p->ng, p->n_sm, s);
  if (st != BSP_OK) return st;
  b.items = p->d_byi;
  st = launch_warp_yfpass(b, p->nbyi, s);
  if (st != BSP_OK) return st;
  b.items = p->d_bxi;
  return launch_warp_xfpass(b, p->nbxi, 1.f, s);
}

bsp_status bsp_grad(bsp_plan* p, const void* spec, const double* dl_db, float* dl_ddelta, void* stream) {
  if (!p || !spec || !dl_db || !dl_ddelta) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (p->prec == BSP_FP64 || p->dim == 2 || p->order == 4)
    return fail(BSP_ERR_NOT_SUPPORTED, "bsp_grad needs a 3D bispectrum plan in FP32 or mixed precision");
  if (!warp_fft_supported(p->ngs) || !warp_fft_supported(p->ng))
    return fail(BSP_ERR_NOT_SUPPORTED, "bsp_grad needs grid sides 2^p or 3 * 2^p in [128, 1024]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bsp_status st = grad_setup(p, s);
  if (st != BSP_OK) return st;
  // W, then the shell fields on the evaluation grid (recomputed: nothing is kept from a forward
  // call), the adjoint products G_n and their forward transforms along z, all at once or, under a
  // memory budget, one x-slab at a time after a single X and Y pass
  st = launch_build_w(dl_db, p->d_cnorm, p->d_w_ptr, p->d_w_idx, p->adj_entries, p->d_w, s);
  if (st != BSP_OK) return st;
  if (p->slab_nx && (st = plan_passes<float>(p, spec, p->fields, s, nullptr, false, kPassXY)) != BSP_OK) return st;
  PassArgs a{};
  a.n_sm = p->n_sm;
  a.g1 = p->g1;
  a.g2 = p->g2;
  a.fields = p->d_grad_spec;
  a.tw = p->tw;
  a.geom = p->d_geom;
  a.ng = p->ng;
  a.ngs = p->ngs;
  a.rsd = p->rsd;
  a.beta = p->beta;
  a.rmax = p->rmax;
  a.stw = p->d_stw;
  a.stw_half = p->d_stw_half;
  for (int k = 0; k < p->n_slabs(); ++k) {
    const int part = p->slab_nx ? k : kPassAll;
    if ((st = plan_passes<float>(p, spec, p->fields, s, nullptr, false, part)) != BSP_OK) return st;
    const long long nvox = (long long)p->slab_len(k) * p->ngs * p->ngs;
    st = launch_adjoint_products(static_cast<const float*>(p->fields), nvox, p->ns, p->adj_np, p->d_adj_pairs,
                                 p->adj_npairs, p->d_w, p->d_gfields, p->n_sm, s);
    if (st != BSP_OK) return st;
    // forward transforms of G_n, kept on each shell's modes: conj(.) K (ng/S)^3 into the ng spectrum
    a.slab_x0 = p->slab_nx ? p->slab_x0(k) : 0;
    a.slab_nx = p->slab_nx ? p->slab_len(k) : 0;
    st = launch_warp_zfpass(a, p->d_gfields, (long long)p->ns * p->slab_len(k) * p->ngs, p->n_sm, s);
    if (st != BSP_OK) return st;
  }
  a.slab_x0 = a.slab_nx = 0;
  a.items = p->d_wyi;
  st = launch_warp_yfpass(a, p->nwyi, s);
  if (st != BSP_OK) return st;
  a.items = p->d_wxi;
  st = launch_warp_xfpass(a, p->nwxi, (float)p->sum_scale, s);
  if (st != BSP_OK) return st;
  // one pruned inverse transform of the whole ball on the ng grid
  PassArgs b{};
  b.n_sm = p->n_sm;
  b.spec = p->d_grad_spec;
  b.g1 = p->g1b;
  b.g2 = p->g2b;
  b.fields = dl_ddelta;
  b.tw = p->d_tw_ng;
  b.geom = p->d_ball;
  b.ng = p->ng;
  b.ngs = p->ng;
  b.rsd = 0;
  b.beta = 0.0;
  b.rmax = (int)isqrt_ll(p->q[p->ns] - 1) + 1;
  b.stw = p->d_stw_ng;
  b.stw_half = p->d_stw_ng_half;
  b.items = p->d_bxi;
  st = launch_warp_xpass(b, p->nbxi, s);
  if (st != BSP_OK) return st;
  b.items = p->d_byi;
  st = launch_warp_ypass(b, p->nbyi, s);
  if (st != BSP_OK) return st;
  return launch_warp_zpass(b, (long long)p->ng * p->ng, p->n_sm, s);
}

bsp_status bsp_last_sums(const bsp_plan* p, const double** msum) {
  if (!p || !msum) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  *msum = p->msum;
  return BSP_OK;
}

}  // extern "C"
