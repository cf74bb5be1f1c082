// C ABI of the bispectrum library: error reporting, the estimator (Eqs. (2.7)-(2.11)) and the
// (mu, t) map (Eq. (2.4)), batches, the host entry, the adjoint and timing. The plan itself is
// built in bispec_plan.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "plan_internal.h"

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
      a.np = L.np;
      a.kt = L.kt;
      a.groups = L.d_tc_groups;
      a.n_tg = L.n_tg;
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
    const bool work = p->prec == BSP_MIXED_BF16X3 ? L.n_tg > 0 : L.ntiles > 0;
    const bool sampled = !L.top && !(p->prec == BSP_MIXED_BF16X3 && p->n_zlev > 0);  // else the Z pass did it
    n += sampled + (p->prec == BSP_MIXED_BF16X3 ? 1 : 2) * work;
  }
  return n + (p->prec == BSP_MIXED_BF16X3 ? 1 : 0);  // one cross-block sum for all tensor-core levels
}

// The contraction of x-slab k of an x-slab plan (one level, the evaluation grid) on the slab's
// fields in p->fields, its sums added to msum after the first slab.
template <typename T>
bsp_status contract_slab(bsp_plan* p, int k, cudaStream_t s) {
  if (p->levels.empty()) return BSP_OK;
  const ContractLevel& L = p->levels[0];
  if (p->prec == BSP_MIXED_BF16X3) {
    // the slab's split fields through the full-slab or last-slab tensor map, a fixed number of
    // voxel blocks (blocks past the slab's voxels write zero sums), sums added over the slabs
    if (L.n_tg == 0) return BSP_OK;
    const long long nvox = (long long)p->slab_len(k) * p->ngs * p->ngs;
    const long long chunks = nvox / kTcVoxelChunk;
    TcArgs a{};
    a.nvox = nvox;
    a.np = L.np;
    a.kt = L.kt;
    a.groups = L.d_tc_groups;
    a.n_tg = L.n_tg;
    a.gridy = L.gridy;
    a.vox_per_block = ((chunks + L.gridy - 1) / L.gridy) * kTcVoxelChunk;
    a.partial = L.tc_partial;
    a.error = p->d_error;
    const bool last = k == p->n_slabs() - 1 && p->slab_len(k) != p->slab_len(0);
    bsp_status st = launch_contract_tc(a, last ? &L.tmap_last : &L.tmap, s);
    if (st != BSP_OK) return st;
    return launch_reduce_tc_all(p->d_tc_bins, (int)p->trips.size(), p->msum, s, k > 0);
  }
  if (L.ntiles == 0) return BSP_OK;
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
      // split fields of the slab: [2][ns][slab planes x S^2]
      if (split) a.split_lo = (long long)p->ns * a.slab_nx * p->ngs * p->ngs / 2;
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
    st = plan_passes<T>(p, spec, p->fields, s, rec ? ev + 1 : nullptr, split, kPassXY);
    if (st != BSP_OK) return st;
    for (int k = 0; k < p->n_slabs(); ++k) {
      if ((st = plan_passes<T>(p, spec, p->fields, s, nullptr, split, k)) != BSP_OK) return st;
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
      const bool work = !p->levels.empty() && (split ? p->levels[0].n_tg > 0 : p->levels[0].ntiles > 0);
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
  // contraction levels, each pair on its smallest exact grid (a split-BF16 plan may contract some
  // pairs on a larger level where that is faster; that extra work is not counted): fields read
  // once per level (lower levels also read their samples of the evaluation grid and write them),
  // work per level on its g^3 grid
  for (const auto& lv : p->exact_levels) {
    const int g = lv.first;
    const std::vector<int>& bins = lv.second;
    const bool top = g == p->ngs;
    const double nv = p->dim == 2 ? (double)g * g : (double)g * g * g;
    int nsh = 0;
    if (top) {
      nsh = p->ns + p->n_extra();
    } else {
      std::vector<char> used(p->ns, 0);
      for (int b : bins) used[p->trips[b].a] = used[p->trips[b].b] = used[p->trips[b].c] = 1;
      for (char u : used) nsh += u;
    }
    long long npairs = 0;
    for (size_t i = 0; i < bins.size(); ++i) {
      const bsp_triplet& a = p->trips[bins[i]];
      if (i == 0 || a.a != p->trips[bins[i - 1]].a || a.b != p->trips[bins[i - 1]].b) npairs += 1;
    }
    bytes[BSP_STAGE_CONTRACT] += re * nsh * nv * (top ? 1.0 : 3.0);
    if (p->prec == BSP_MIXED_BF16X3)  // split-BF16 GEMM over the padded shell columns
      flops[BSP_STAGE_CONTRACT] += 3.0 * 2.0 * (double)npairs * (double)tc_padded_shells(nsh) * nv;
    else
      flops[BSP_STAGE_CONTRACT] += ((double)npairs + 2.0 * (double)bins.size()) * nv;
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

template bsp_status plan_passes<float>(bsp_plan*, const void*, void*, cudaStream_t, cudaEvent_t*, bool, int);
template bsp_status plan_passes<double>(bsp_plan*, const void*, void*, cudaStream_t, cudaEvent_t*, bool, int);

}  // namespace bsp

extern "C" {

const char* bsp_last_error(void) { return g_error; }

const char* bsp_version(void) { return "bispec-gb300 0.1 (sm_103a)"; }

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
    if (p->slab_nx)
      return fail(BSP_ERR_NOT_SUPPORTED, "bsp_contract: a split-BF16 plan under a memory budget holds one x-slab of fields");
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
  if (flag) {
    // reported once: later checks report only later give-ups
    BSP_CUDA(cudaMemset(p->d_error, 0, sizeof(int)));
    return fail(BSP_ERR_TIMEOUT, "a bounded device-side wait gave up in an earlier call");
  }
  return BSP_OK;
}

bsp_status bsp_selftest_wait_timeout(bsp_plan* p, void* stream) {
  if (!p) return fail(BSP_ERR_INVALID_ARG, "plan is NULL");
  return launch_wait_selftest(p->d_error, static_cast<cudaStream_t>(stream));
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
