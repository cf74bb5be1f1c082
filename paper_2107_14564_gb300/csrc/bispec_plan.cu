// Plan construction (Sec. 2.1 binning, the evaluation grid and contraction levels, Eq. (2.10)
// counts on the GPU in FP64, labels of Eq. (2.4), autotuning) and the plan's query entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "plan_internal.h"

namespace bsp {

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
                const std::vector<int>* ids) {
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

// Pair groups of the tensor-core contraction (see TcArgs). A slot holds three fields f0, f1, f2
// and the flag s; its pairs are (f0, s ? f1 : f0) in tile 0, (f0, f2) in tile 1 and (f1, f2) in
// tile 2 of its tile group, so one generator thread forms KT pair products from three loaded
// fields. Every tile of a tile group costs the same MMAs, so the grouping minimises tiles (tile
// groups x KT) and, at equal cost, takes the larger KT (fewer field loads per pair).
//
// Groups are chosen greedily and deterministically: the uncovered pair whose best candidate group
// covers the fewest uncovered pairs (then: has the fewest such candidates) is covered next, by
// its candidate that covers the most uncovered pairs and, among those, leaves the easiest pairs
// for later (lowest sum of their best scores).
namespace {
struct Grp {
  int f0, f1, f2, s;
};
void grp_pairs(const Grp& g, int2 out[3]) {
  out[0] = make_int2(g.f0, g.s ? g.f1 : g.f0);
  out[1] = make_int2(g.f0, g.f2);
  out[2] = make_int2(g.f1, g.f2);
}
}  // namespace

TcGrouping group_pairs(const std::vector<int2>& pairs, int nf, int kt_max) {
  const int np = (int)pairs.size();
  std::vector<int> id((size_t)nf * nf, -1);
  for (int i = 0; i < np; ++i) {
    id[(size_t)pairs[i].x * nf + pairs[i].y] = i;
    id[(size_t)pairs[i].y * nf + pairs[i].x] = i;
  }
  auto pid = [&](int2 q) { return id[(size_t)q.x * nf + q.y]; };
  // greedy cover with groups of kt pairs
  auto cover = [&](int kt) {
    std::vector<Grp> groups;
    std::vector<char> unc(np, 1);
    int left = np;
    // distinct uncovered pairs a group covers in its first kt tiles
    auto score = [&](const Grp& g) {
      int2 q[3];
      grp_pairs(g, q);
      int ids[3], n = 0;
      for (int j = 0; j < kt; ++j) {
        const int k = pid(q[j]);
        if (k < 0 || !unc[k]) continue;
        bool dup = false;
        for (int t = 0; t < n; ++t) dup |= ids[t] == k;
        if (!dup) ids[n++] = k;
      }
      return n;
    };
    auto cands = [&](int i, std::vector<Grp>& out) {
      out.clear();
      const int a = pairs[i].x, b = pairs[i].y;
      const int xs[2][2] = {{a, b}, {b, a}};
      for (int o = 0; o < (a == b ? 1 : 2); ++o) {
        const int x = xs[o][0], y = xs[o][1];
        for (int f = 0; f < nf; ++f) out.push_back({x, y, f, 1});  // tile 0 (f0, f1)
        for (int f = 0; f < nf; ++f) {                              // tile 1 (f0, f2)
          out.push_back({x, f, y, 1});
          if (kt >= 3 || f == 0) out.push_back({x, kt >= 3 ? f : x, y, 0});  // f1 unused at kt 2
        }
        if (kt >= 3)
          for (int f = 0; f < nf; ++f)                              // tile 2 (f1, f2)
            for (int s = 0; s < 2; ++s) out.push_back({f, x, y, s});
      }
      if (a == b) {                                                 // tile 0 (f0, f0)
        for (int f2 = 0; f2 < nf; ++f2)
          for (int f1 = 0; f1 < (kt >= 3 ? nf : 1); ++f1) out.push_back({a, kt >= 3 ? f1 : a, f2, 0});
      }
    };
    std::vector<Grp> cs;
    std::vector<int> best(np, 0);
    while (left > 0) {
      int pick = -1, pick_m = 0, pick_cnt = 0;
      for (int i = 0; i < np; ++i) {
        if (!unc[i]) continue;
        cands(i, cs);
        int m = 0, cnt = 0;
        for (const Grp& g : cs) {
          const int sc = score(g);
          if (sc > m) { m = sc; cnt = 1; } else if (sc == m) { ++cnt; }
        }
        best[i] = m;
        if (pick < 0 || m < pick_m || (m == pick_m && cnt < pick_cnt)) { pick = i; pick_m = m; pick_cnt = cnt; }
      }
      cands(pick, cs);
      Grp chosen = cs[0];
      long long chosen_h = -1;
      for (const Grp& g : cs) {
        if (score(g) != pick_m) continue;
        int2 q[3];
        grp_pairs(g, q);
        long long h = 0;
        for (int j = 0; j < kt; ++j) {
          const int k = pid(q[j]);
          if (k >= 0 && unc[k]) h += best[k];
        }
        if (chosen_h < 0 || h < chosen_h) { chosen = g; chosen_h = h; }
      }
      int2 q[3];
      grp_pairs(chosen, q);
      for (int j = 0; j < kt; ++j) {
        const int k = pid(q[j]);
        if (k >= 0 && unc[k]) { unc[k] = 0; --left; }
      }
      groups.push_back(chosen);
    }
    return groups;
  };
  // candidate groupings: one pair per slot, or greedy groups of 2 and 3
  std::vector<Grp> best_groups;
  int best_kt = 1;
  for (int i = 0; i < np; ++i) best_groups.push_back({pairs[i].x, pairs[i].y, pairs[i].x, 1});
  long long best_cost = (np + kTcSlots - 1) / kTcSlots;
  if (np > kTcSlots) {
    for (int kt = 2; kt <= kt_max; ++kt) {
      std::vector<Grp> g = cover(kt);
      const long long cost = (long long)kt * (((long long)g.size() + kTcSlots - 1) / kTcSlots);
      if (cost <= best_cost) { best_cost = cost; best_kt = kt; best_groups.swap(g); }
    }
  }
  // Slot order: a generator's 8-byte shared-memory load of field slot f is served in half-warp
  // phases of 4 consecutive slots, each slot's quad reading the 32-byte segment (K ^ (n >> 1)) & 3
  // of field n's swizzled 128-byte row (K the K step). A phase is conflict-free when, for every
  // field slot, its 4 slots read equal fields or fields with distinct (n >> 1) & 3. Phases are
  // filled greedily, each group in the first of its equivalent field orders that fits (a triangle
  // may permute its three fields, a group of two its last two, a single pair its two); slots a
  // phase cannot fill without a conflict take the next group as it is, and padding slots repeat
  // a group of their phase (a broadcast) with the active flag clear.
  const int nfld = best_kt == 1 ? 2 : 3;
  auto orders = [&](const Grp& g, std::vector<Grp>& out) {
    out.clear();
    out.push_back(g);
    if (!g.s) return;
    if (best_kt == 1) {
      out.push_back({g.f1, g.f0, g.f1, 1});
    } else if (best_kt == 2) {
      out.push_back({g.f0, g.f2, g.f1, 1});
    } else {
      const int f[3] = {g.f0, g.f1, g.f2};
      const int perm[5][3] = {{0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
      for (auto& p : perm) out.push_back({f[p[0]], f[p[1]], f[p[2]], 1});
    }
  };
  auto fld = [](const Grp& g, int f) { return f == 0 ? g.f0 : f == 1 ? g.f1 : g.f2; };
  std::vector<Grp> placed;  // in slot order; (-1, ...) marks padding
  {
    std::vector<Grp> rest = best_groups, ords;
    while (!rest.empty()) {
      int used[3][4];
      for (auto& u : used) for (int& x : u) x = -1;
      int n = 0;
      for (size_t k = 0; k < rest.size() && n < 4;) {
        orders(rest[k], ords);
        bool put = false;
        for (const Grp& o : ords) {
          bool ok = true;
          for (int f = 0; f < nfld && ok; ++f) {
            const int v = fld(o, f), b = (v >> 1) & 3;
            ok = used[f][b] < 0 || used[f][b] == v;
          }
          if (!ok) continue;
          for (int f = 0; f < nfld; ++f) used[f][(fld(o, f) >> 1) & 3] = fld(o, f);
          placed.push_back(o);
          put = true;
          break;
        }
        if (put) { rest.erase(rest.begin() + (long)k); ++n; } else { ++k; }
      }
      if (n == 0) { placed.push_back(rest.front()); rest.erase(rest.begin()); ++n; }
      const bool last = rest.empty();
      // a phase that could not be completed without conflicts takes the next groups as they are
      while (n < 4 && !rest.empty() && !last) { placed.push_back(rest.front()); rest.erase(rest.begin()); ++n; }
      while (n < 4) { placed.push_back({-1, 0, 0, 0}); ++n; }
    }
  }
  TcGrouping out;
  out.kt = best_kt;
  const int nslots = (int)placed.size();
  out.n_tg = np == 0 ? 0 : (nslots + kTcSlots - 1) / kTcSlots;
  out.slots.assign((size_t)out.n_tg * kTcSlots, make_int4(0, 0, 0, 0));
  out.where.assign(np, -1);
  for (int g = 0; g < nslots; ++g) {
    const int ph0 = g - g % 4;
    if (placed[g].f0 < 0) {  // padding: repeat the phase's first group, inactive
      const Grp& r = placed[ph0];
      out.slots[g] = make_int4(r.f0, r.f1, r.f2, r.s ? 1 : 0);
      continue;
    }
    const Grp& gr = placed[g];
    out.slots[g] = make_int4(gr.f0, gr.f1, gr.f2, (gr.s ? 1 : 0) | 2);
    int2 q[3];
    grp_pairs(gr, q);
    const int tg = g / kTcSlots, slot = g % kTcSlots;
    for (int j = 0; j < out.kt; ++j) {
      const int k = pid(q[j]);
      if (k >= 0 && out.where[k] < 0) out.where[k] = (tg * out.kt + j) * kTcSlots + slot;
    }
  }
  return out;
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
    if (p->prec == BSP_MIXED_BF16X3 && !(p->dim == 3 && warp_fft_supported(p->ngs)))
      return fail(BSP_ERR_NOT_SUPPORTED,
                  "mem_budget_bytes below the shell fields of a split-BF16 plan on an evaluation grid the warp passes do not handle");
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
// kernel on the plan's own buffers with the voxel range of each tile group split over m x (SM
// count) blocks, m in kTuneMults (fewer when the level has fewer 64-voxel chunks), 3 launches after one
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
    if (L.n_tg == 0) continue;
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
      a.np = L.np;
      a.kt = L.kt;
      a.groups = L.d_tc_groups;
      a.n_tg = L.n_tg;
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
    // a plan streaming x-slabs holds one slab's fields: its Z pass is timed on the first slab
    const int part = !p->slab_nx ? kPassAll : pass == 0 ? kPassXY : 0;
    if (p->slab_nx && (st = plan_passes<float>(p, spec, p->fields, s, nullptr, split, kPassXY)) != BSP_OK) break;
    for (int m : mults) {
      *knob[pass] = m * p->n_sm;
      // warm-up (the Y pass needs the X pass output once; the Z pass reads what Y wrote)
      if ((st = plan_passes<float>(p, spec, p->fields, s, nullptr, split, part)) != BSP_OK) break;
      if ((ce = cudaEventRecord(e0, s)) != cudaSuccess) { st = cuda_fail(ce, "cudaEventRecord"); break; }
      for (int r = 0; r < 3 && st == BSP_OK; ++r) st = plan_passes<float>(p, spec, p->fields, s, nullptr, split, part);
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

// Cost model of one tensor-core contraction level, in microseconds on the whole GPU: every
// tile group of the level costs, per 64-voxel chunk on one SM, kTcChunkCycles[KT - 1] cycles
// (NP = 32 padded shells; twice that at NP = 64) whatever number of its 64 slots hold pairs;
// a level also costs a fixed launch, pipeline fill and flush time, and a level below the
// evaluation grid the Z pass's writes of its split fields (4 bytes per shell and voxel). The
// per-chunk cycles are measured per-SM times of levels with one tile group of KT = 1 (900-935
// cycles on 192^3 .. 768^3 grids) and KT = 3 (1133-1174 cycles on 384^3 and 768^3) on a GB300 at
// 2070 MHz, KT = 2 between them. The level-field writes are charged at half the copy bandwidth:
// an Ng = 768 Z pass writing 7.5 GB of level fields beside 43.5 GB of evaluation-grid fields took
// 19.7 ms, the same fields written x-slab by x-slab without them 14.9 ms.
namespace {
constexpr double kTcChunkCycles[3] = {925.0, 1040.0, 1150.0};
constexpr double kTcLevelFixedUs = 4.0;
constexpr double kTcSmMhz = 2070.0;
constexpr double kTcFieldBytesPerUs = 3.4e6;

double tc_level_cost_us(const bsp_plan* p, int g, const std::vector<int>& bins) {
  const bool top = g == p->ngs;
  std::vector<int> loc(p->ns, -1);
  int nsh = 0;
  if (top) {
    for (int n = 0; n < p->ns; ++n) loc[n] = nsh++;
  } else {
    std::vector<char> used(p->ns, 0);
    for (int b : bins) used[p->trips[b].a] = used[p->trips[b].b] = used[p->trips[b].c] = 1;
    for (int n = 0; n < p->ns; ++n)
      if (used[n]) loc[n] = nsh++;
  }
  std::vector<int2> pairs;
  for (size_t i = 0; i < bins.size(); ++i) {
    const bsp_triplet& t = p->trips[bins[i]];
    if (i == 0 || t.a != p->trips[bins[i - 1]].a || t.b != p->trips[bins[i - 1]].b)
      pairs.push_back(make_int2(loc[t.a], loc[t.b]));
  }
  const int np = tc_padded_shells(nsh);
  const TcGrouping G = group_pairs(pairs, nsh, np == 32 ? 3 : 2);
  const double vox = (double)g * g * g;
  const double chunks_per_sm = std::ceil(vox / kTcVoxelChunk / std::max(1, p->n_sm));
  const double cyc = kTcChunkCycles[std::min(std::max(G.kt, 1), 3) - 1] * (np / 32.0);
  double us = kTcLevelFixedUs + chunks_per_sm * G.n_tg * cyc / kTcSmMhz;
  if (!top) us += (double)nsh * vox * 4.0 / kTcFieldBytesPerUs;
  return us;
}
}  // namespace

// Merging of tensor-core contraction levels: a level whose pairs fit into the spare slots (or a
// larger KT) of the next level up can cost less there than on its own smaller grid, because a
// level's time follows its tile groups, not its pairs. Levels are merged bottom-up, each into
// the next level, while the model above says the sum of the two costs more than the merged
// level. A pair's evaluation grid stays exact on any larger divisor grid, so a merge changes
// only the order of the additions in a bin's sum.
void merge_tc_levels(const bsp_plan* p, std::vector<std::pair<int, std::vector<int>>>& by_g) {
  size_t i = 0;
  while (i + 1 < by_g.size()) {
    std::vector<int> u = by_g[i].second;
    u.insert(u.end(), by_g[i + 1].second.begin(), by_g[i + 1].second.end());
    std::sort(u.begin(), u.end());
    const double apart = tc_level_cost_us(p, by_g[i].first, by_g[i].second) +
                         tc_level_cost_us(p, by_g[i + 1].first, by_g[i + 1].second);
    const double merged = tc_level_cost_us(p, by_g[i + 1].first, u);
    if (merged < apart) {
      by_g[i + 1].second.swap(u);
      by_g.erase(by_g.begin() + (long)i);
    } else {
      ++i;
    }
  }
}

// Contraction levels (see ContractLevel): each pair (a, b) of the kept bins goes to the smallest
// divisor g of the evaluation grid (g % 8 == 0, g >= 16) above r_a + r_b + r_cmax - 3, the largest
// wavevector component of its triple products; split-BF16 plans then merge levels where the
// cost model above favours it.
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
  p->exact_levels = by_g;
  if (p->prec == BSP_MIXED_BF16X3) merge_tc_levels(p, by_g);
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
      const TcGrouping G = group_pairs(pairs, nsh, L.np == 32 ? 3 : 2);
      L.kt = G.kt;
      L.n_tg = G.n_tg;
      std::vector<int> tmap(L.bins.size());
      int pi = -1;
      for (size_t i = 0; i < L.bins.size(); ++i) {
        if (i == 0 || la[i] != la[i - 1] || lb[i] != lb[i - 1]) ++pi;
        if (G.where[pi] < 0) return fail(BSP_ERR_CUDA, "internal: a pair of the contraction has no slot");
        tmap[i] = G.where[pi] * L.np + lc[i];
      }
      // under a memory budget the level is contracted slab by slab over the slab's voxels
      const long long cvox = p->slab_nx ? (long long)p->slab_len(p->n_slabs() - 1) * S * S : L.nvox();
      const long long chunks = cvox / kTcVoxelChunk;
      long long gy = std::min<long long>(std::max(1, p->n_sm), chunks);
      L.vpb = ((chunks + gy - 1) / gy) * kTcVoxelChunk;
      L.gridy = p->slab_nx ? (int)gy : (int)((L.nvox() + L.vpb - 1) / L.vpb);
      // partial sums sized for the largest split the autotuner may pick
      const long long gmax = p->autotune ? std::min<long long>((long long)kTuneMults[kNumTune - 1] * std::max(1, p->n_sm), chunks) : gy;
      L.gridy_cap = p->slab_nx ? L.gridy  // every slab runs L.gridy blocks
                               : (int)((L.nvox() + ((chunks + gmax - 1) / gmax) * kTcVoxelChunk - 1) /
                                       (((chunks + gmax - 1) / gmax) * kTcVoxelChunk));
      if ((st = dev_upload(p, G.slots, &L.d_tc_groups, s)) != BSP_OK) return st;
      L.tc_off = tmap;
      if ((st = dev_alloc(p, tc_partial_entries(std::max(L.n_tg, 1), std::max(L.kt, 1), std::max(L.gridy, L.gridy_cap), L.np) * sizeof(float2), &tmp)) != BSP_OK)
        return st;
      L.tc_partial = static_cast<float2*>(tmp);
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
    if (p->prec == BSP_MIXED_BF16X3 && L.n_tg > 0 && p->slab_nx) {
      // one x-slab's split fields [2][ns][slab planes x S^2]: a full slab and the last one
      st = encode_split_map(&L.tmap, p->fields, (long long)p->slab_len(0) * S * S, nsh, L.np);
      if (st == BSP_OK)
        st = encode_split_map(&L.tmap_last, p->fields, (long long)p->slab_len(p->n_slabs() - 1) * S * S, nsh, L.np);
      if (st != BSP_OK) return st;
    } else if (p->prec == BSP_MIXED_BF16X3 && L.n_tg > 0) {
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
  if (p->prec == BSP_MIXED_BF16X3 && p->autotune && !p->slab_nx) {
    if ((st = autotune_levels(p, s)) != BSP_OK) return st;
  }
  if (p->prec == BSP_MIXED_BF16X3) {
    std::vector<TcBin> tb(p->trips.size());
    for (const ContractLevel& L : p->levels)
      for (size_t i = 0; i < L.bins.size(); ++i) {
        TcBin& b = tb[L.bins[i]];
        b.partial = L.tc_partial;
        b.stride = (long long)L.n_tg * L.kt * kTcSlots * L.np;
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

}  // namespace bsp

extern "C" {

bsp_status bsp_plan_create(const bsp_plan_desc* desc, void* stream, bsp_plan** out) {
  if (!out) return fail(BSP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  set_error_c("");
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

bsp_status bsp_plan_bin_levels(const bsp_plan* p, int n, int* level, int* slot) {
  if (!p) return fail(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n != (int)p->trips.size()) return fail(BSP_ERR_INVALID_ARG, "n must be the number of kept bins");
  for (int l = 0; l < (int)p->levels.size(); ++l) {
    const ContractLevel& L = p->levels[l];
    for (size_t i = 0; i < L.bins.size(); ++i) {
      if (level) level[L.bins[i]] = l;
      if (slot) slot[L.bins[i]] = p->prec == BSP_MIXED_BF16X3 && L.np > 0 ? L.tc_off[i] / L.np : -1;
    }
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

}  // extern "C"
