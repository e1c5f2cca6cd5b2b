// Host construction of the HDD plan: decomposition tree (Sec. 2.1), index sets
// I(gamma), I(d omega) (Sec. 2.1), extend-add maps of the father system
// (Sec. 3.3, Eq. block_equation4), the pruned descent set (Sec. 5.3), the
// per-height launch schedule and the lifetime-packed Schur arena.
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>

#include "plan.h"

namespace hdd {

namespace {

bool unknown(int N, int i, int j) { return i >= 1 && j >= 1 && i <= N - 2 && j <= N - 2; }

// Binary tree: split the longer side at the cell-aligned midpoint (x on ties),
// stop when both sides are at most `leaf` cells.
void build_tree(Plan& p) {
  const int N = p.N;
  p.nodes.clear();
  Node root;
  root.x0 = 0; root.x1 = N - 1; root.y0 = 0; root.y1 = N - 1;
  p.nodes.push_back(root);
  std::vector<int> stack{0};
  while (!stack.empty()) {
    int k = stack.back();
    stack.pop_back();
    Node nd = p.nodes[k];
    int w = nd.x1 - nd.x0, hgt = nd.y1 - nd.y0;
    if (w <= p.leaf && hgt <= p.leaf) continue;
    Node a = nd, b = nd;
    a.depth = b.depth = nd.depth + 1;
    a.parent = b.parent = k;
    a.gamma.clear(); b.gamma.clear();
    a.child[0] = a.child[1] = b.child[0] = b.child[1] = -1;
    a.split = b.split = 0;
    if (w >= hgt) {
      int xm = nd.x0 + w / 2;
      a.x1 = xm; b.x0 = xm;
      p.nodes[k].split = 'x'; p.nodes[k].cut = xm;
    } else {
      int ym = nd.y0 + hgt / 2;
      a.y1 = ym; b.y0 = ym;
      p.nodes[k].split = 'y'; p.nodes[k].cut = ym;
    }
    int base = (int)p.nodes.size();
    p.nodes.push_back(a);
    p.nodes.push_back(b);
    p.nodes[k].child[0] = base;
    p.nodes[k].child[1] = base + 1;
    stack.push_back(base + 1);
    stack.push_back(base);
  }
  // index sets
  for (Node& nd : p.nodes) {
    nd.bnd.clear();
    nd.gamma.clear();
    for (int j = nd.y0; j <= nd.y1; ++j)
      for (int i = nd.x0; i <= nd.x1; ++i) {
        bool edge = (i == nd.x0 || i == nd.x1 || j == nd.y0 || j == nd.y1);
        if (edge && unknown(N, i, j)) nd.bnd.push_back(j * N + i);
      }
    if (nd.leaf()) {
      for (int j = nd.y0 + 1; j < nd.y1; ++j)
        for (int i = nd.x0 + 1; i < nd.x1; ++i) nd.gamma.push_back(j * N + i);
    } else if (nd.split == 'x') {
      for (int j = nd.y0 + 1; j < nd.y1; ++j) nd.gamma.push_back(j * N + nd.cut);
    } else {
      for (int i = nd.x0 + 1; i < nd.x1; ++i) nd.gamma.push_back(nd.cut * N + i);
    }
    nd.m = (int)nd.gamma.size();
    nd.b = (int)nd.bnd.size();
    nd.nf = nd.m + nd.b + 1;
  }
  // heights (children have larger indices than their parent)
  for (int k = (int)p.nodes.size() - 1; k >= 0; --k) {
    Node& nd = p.nodes[k];
    nd.height = nd.leaf() ? 0 : 1 + std::max(p.nodes[nd.child[0]].height, p.nodes[nd.child[1]].height);
  }
}

}  // namespace

std::string build_plan(const hdd_plan_desc& d, Plan& p) {
  if (d.N < 3) return "N must be >= 3";
  if (d.N > 8193) return "N must be <= 8193";
  if (d.leaf < 1) return "leaf must be >= 1";
  if (d.n_z < 1 || d.n_z > 256) return "n_z must be in 1..256";
  if (d.n_obs < 1) return "n_obs must be >= 1";
  if (!d.obs_vertex) return "obs_vertex is NULL";
  if (!(d.sigma > 0.0)) return "sigma must be > 0";
  if (d.precision != HDD_FP64 && d.precision != HDD_MIXED_FP32) return "unknown precision";
  if (d.ir_max_iter < 0 || d.ir_max_iter > 64) return "ir_max_iter must be in 0..64";
  if (d.fp64_top_levels < 0 || d.fp64_top_levels > 64) return "fp64_top_levels must be in 0..64";
  if (d.fuse_height < 0 || d.fuse_height > kFuseMaxHeight) return "fuse_height must be in 0..6";
  p.N = d.N; p.leaf = d.leaf; p.n_z = d.n_z; p.n_obs = d.n_obs;
  p.n_t = 2 * (d.N - 1) * (d.N - 1);
  p.f = d.f; p.sigma = d.sigma; p.h = 1.0 / (d.N - 1);
  p.precision = d.precision; p.ir_max_iter = d.ir_max_iter; p.ir_tol = d.ir_tol;
  p.fp64_top_levels = d.fp64_top_levels;
  p.fuse_height = d.fuse_height;
  p.device = d.device;
  if (d.obs_kind != HDD_OBS_VERTEX && d.obs_kind != HDD_OBS_MEANS) return "unknown obs_kind";
  p.obs_kind = d.obs_kind;
  if (p.obs_kind == HDD_OBS_VERTEX) {
    p.obs.assign(d.obs_vertex, d.obs_vertex + d.n_obs);
    for (int v : p.obs) {
      if (v < 0 || v >= d.N * d.N) return "observation vertex out of range";
      if (!unknown(d.N, v % d.N, v / d.N)) return "observation vertex on the Dirichlet boundary";
    }
  }

  build_tree(p);
  const int N = p.N;
  const int nn = (int)p.nodes.size();

  if (p.obs_kind == HDD_OBS_MEANS) {
    // observations are node means; the vertices whose values they need are the
    // boundary unknowns of the observed nodes (their owners are the ancestors, so
    // the pruned descent below visits exactly the ancestors, Sec. 5.2 Remark b)
    p.obs_nodes.assign(d.obs_vertex, d.obs_vertex + d.n_obs);
    std::vector<char> seen((size_t)N * N, 0);
    for (int k : p.obs_nodes) {
      if (k < 0 || k >= nn) return "observed node out of range";
      for (int v : p.nodes[k].bnd)
        if (!seen[v]) { seen[v] = 1; p.obs.push_back(v); }
    }
    std::sort(p.obs.begin(), p.obs.end());
    if (p.obs.empty()) p.obs = p.nodes[0].gamma;   // only Omega observed: the root's interface
  }
  p.n_conv = (int)p.obs.size();

  // owner of every unknown: each is eliminated exactly once
  p.owner.assign((size_t)N * N, -1);
  for (int k = 0; k < nn; ++k)
    for (int v : p.nodes[k].gamma) {
      if (p.owner[v] != -1) return "internal: vertex eliminated twice";
      p.owner[v] = k;
    }
  for (int j = 1; j <= N - 2; ++j)
    for (int i = 1; i <= N - 2; ++i)
      if (p.owner[j * N + i] < 0) return "internal: vertex never eliminated";

  // pruned descent: root-to-owner paths of the observations (Sec. 5.3)
  for (int v : p.obs) {
    int k = p.owner[v];
    while (k >= 0 && !p.nodes[k].visited) {
      p.nodes[k].visited = true;
      k = p.nodes[k].parent;
    }
  }

  // precision per node: mixed plans factorise the top fp64_top_levels depths in FP64
  for (Node& nd : p.nodes) nd.fp64 = (p.precision == HDD_FP64) || nd.depth < p.fp64_top_levels;

  // fused bottom subtrees: complete subtrees of one precision whose whole
  // elimination fits the shared memory of one CTA (two level buffers of Schur
  // squares + the fronts of the warp groups); the largest such height wins
  p.fuse_soff.assign(nn, 0);
  for (int prec = 0; prec < 2; ++prec) {
    const bool want64 = prec == 0;
    const size_t esz = want64 ? 8 : 4;
    Plan::Fusion best;
    for (int H = p.fuse_height; H >= 1 && best.height == 0; --H) {
      Plan::Fusion fu;
      fu.height = H;
      bool any = false, fits = true;
      for (int k = 0; k < nn && fits; ++k) {
        const Node& r = p.nodes[k];
        if (r.height != H || r.fp64 != want64) continue;
        // complete subtree: every node at height h > 0 has two sons at height h - 1
        std::vector<std::vector<int>> lev(H + 1);
        lev[H].push_back(k);
        bool complete = true;
        for (int hh = H; hh > 0 && complete; --hh)
          for (int q : lev[hh]) {
            const Node& nd = p.nodes[q];
            if (nd.leaf()) { complete = false; break; }
            for (int cidx = 0; cidx < 2; ++cidx) {
              const Node& ch = p.nodes[nd.child[cidx]];
              if (ch.height != hh - 1 || ch.fp64 != want64) complete = false;
              lev[hh - 1].push_back(nd.child[cidx]);
            }
          }
        if (!complete) continue;
        for (int q : lev[0])
          if (!p.nodes[q].leaf()) complete = false;
        if (!complete) continue;
        any = true;
        int32_t desc[12] = {0};
        desc[0] = (int32_t)fu.nodes.size();
        desc[1] = H + 1;
        for (int hh = 0; hh <= H; ++hh) {
          desc[2 + hh] = (int32_t)fu.nodes.size() - desc[0];
          int off = 0, maxk = 0;
          for (int q : lev[hh]) {
            fu.nodes.push_back(q);
            const Node& nd = p.nodes[q];
            if (hh < H) {
              p.fuse_soff[q] = off;
              off += ((nd.b + 1) * (nd.b + 1) + 3) & ~3;
            }
            int ld = (nd.nf + 3) & ~3;
            if ((ld & 7) == 0) ld += 4;
            maxk = std::max(maxk, ((nd.nf * ld) + 3) & ~3);
          }
          fu.sbuf_elems = std::max(fu.sbuf_elems, off);
          const int nh = (int)lev[hh].size();
          int wpf = std::max(1, 16 / nh);
          while (wpf & (wpf - 1)) wpf &= wpf - 1;
          const int ngroups = 16 / wpf;
          int maxnf = 0;
          for (int q : lev[hh]) maxnf = std::max(maxnf, p.nodes[q].nf);
          if (!(wpf == 1 && maxnf <= kTinyMax)) fu.front_elems = std::max(fu.front_elems, ngroups * maxk);
        }
        desc[2 + H + 1] = (int32_t)fu.nodes.size() - desc[0];
        fu.roots.insert(fu.roots.end(), desc, desc + 12);
        fu.smem_bytes = (2 * (size_t)fu.sbuf_elems + (size_t)fu.front_elems) * esz + 64;
        if (fu.smem_bytes > 200 * 1024) fits = false;
      }
      if (any && fits) best = fu;
    }
    if (best.height > 0)
      for (int q : best.nodes) p.nodes[q].fused = true;
    p.fusion[prec] = best;
  }

  // stats, schedule
  p.n_leaves = 0; p.depth = 0; p.n_visited = 0; p.max_front = 0;
  for (const Node& nd : p.nodes) {
    p.n_leaves += nd.leaf();
    p.depth = std::max(p.depth, nd.depth);
    p.n_visited += nd.visited;
    p.max_front = std::max(p.max_front, nd.nf);
  }
  p.height = p.nodes[0].height;
  p.steps.assign(p.height + 1, Step{});
  p.down_visited.assign(p.depth + 1, {});
  p.down_all.assign(p.depth + 1, {});
  p.max_front_small64 = p.max_front_small32 = 0;
  p.max_nf_large = p.max_m_large = p.max_b_large = 0;
  for (int k = 0; k < nn; ++k) {
    Node& nd = p.nodes[k];
    nd.linv = nd.leaf() && !nd.fused && nd.m >= 1 && nd.m <= kLeafInvMax && nd.b <= kLeafInvMaxB;
  }
  for (int k = 0; k < nn; ++k) {
    Node& nd = p.nodes[k];
    if (nd.fused) goto descent_lists;
    if (nd.linv) {
      (nd.fp64 ? p.steps[nd.height].linv64 : p.steps[nd.height].linv32).push_back(k);
      goto descent_lists;
    }
    {
    Step& st = p.steps[nd.height];
    if (nd.fp64) {
      if (nd.nf <= kTinyMax) st.tiny64.push_back(k);
      else if (nd.nf <= kSmallMax64) { st.small64.push_back(k); p.max_front_small64 = std::max(p.max_front_small64, nd.nf); }
      else st.large64.push_back(k);
    } else {
      if (nd.nf <= kTinyMax) st.tiny32.push_back(k);
      else if (nd.nf <= kSmallMax32) { st.small32.push_back(k); p.max_front_small32 = std::max(p.max_front_small32, nd.nf); }
      else st.large32.push_back(k);
    }
    bool large = nd.nf > (nd.fp64 ? kSmallMax64 : kSmallMax32);
    if (large) {
      p.max_nf_large = std::max(p.max_nf_large, nd.nf);
      p.max_m_large = std::max(p.max_m_large, nd.m);
      p.max_b_large = std::max(p.max_b_large, nd.b);
    }
    }
  descent_lists:
    if (nd.m == 0) continue;   // a front with nothing to eliminate has no descent work
    p.down_all[nd.depth].push_back(k);
    if (nd.visited) p.down_visited[nd.depth].push_back(k);
  }

  // factor store and y_g offsets (all nodes keep their factors), in depth-first
  // pre-order (father, son 0's subtree, son 1's subtree), so that every subtree's
  // blocks of one precision are contiguous; y_g blocks padded to four entries
  p.f64_stride = p.f32_stride = 0;
  p.y64_stride = p.y32_stride = 0;
  {
    std::vector<int> todo{0};
    while (!todo.empty()) {
      Node& nd = p.nodes[todo.back()];
      todo.pop_back();
      if (!nd.leaf()) { todo.push_back(nd.child[1]); todo.push_back(nd.child[0]); }
      int64_t& ys = nd.fp64 ? p.y64_stride : p.y32_stride;
      nd.y_off = ys;
      ys += (nd.m + 3) / 4 * 4;
      int64_t sz = nd.linv ? (int64_t)nd.m * (nd.m + 1) / 2 + nd.b : (int64_t)nd.nf * nd.m;
      int64_t& st = nd.fp64 ? p.f64_stride : p.f32_stride;
      nd.f_off = st;
      st += (sz + 31) / 32 * 32;
    }
  }

  // tensor-core staging (large FP32 fronts): lives within one height step
  p.tc_stride = 0;
  for (int hgt = 0; hgt <= p.height; ++hgt) {
    int64_t off = 0;
    for (int k : p.steps[hgt].large32) {
      Node& nd = p.nodes[k];
      const int64_t tiles = (nd.b + kTcTile - 1) / kTcTile, chunks = (nd.m + kTcChunk - 1) / kTcChunk;
      nd.tc_off = off;
      off += tiles * chunks * 2 * kTcBlockBytes;
    }
    p.tc_stride = std::max(p.tc_stride, off);
  }

  // inverted 32 x 32 diagonal blocks of L_gg of the large fronts (POTRF writes
  // them, TRSM applies them): live within one height step
  p.inv_stride = 0;
  for (int hgt = 0; hgt <= p.height; ++hgt) {
    int64_t off = 0;
    for (int prec = 0; prec < 2; ++prec)
      for (int k : (prec ? p.steps[hgt].large32 : p.steps[hgt].large64)) {
        Node& nd = p.nodes[k];
        nd.inv_off = off;
        off += (int64_t)((nd.m + 31) / 32) * 32 * 32 * (nd.fp64 ? 8 : 4);
      }
    p.inv_stride = std::max(p.inv_stride, off);
  }

  // Schur arena: a node's S lives from its own step to its parent's step.
  // Group by the parent's height; first-fit packing of the groups' intervals.
  for (int prec = 0; prec < 2; ++prec) {
    bool want64 = prec == 0;
    struct Region { int start, end; int64_t size, off; std::vector<int> members; };
    std::map<int, Region> regions;   // by parent height
    for (int k = 1; k < nn; ++k) {
      Node& nd = p.nodes[k];
      if (nd.fp64 != want64) continue;
      int H = p.nodes[nd.parent].height;
      auto it = regions.find(H);
      if (it == regions.end()) it = regions.emplace(H, Region{nd.height, H, 0, 0, {}}).first;
      Region& r = it->second;
      r.start = std::min(r.start, nd.height);
      r.members.push_back(k);
      int64_t sz = (int64_t)(nd.b + 1) * (nd.b + 1);
      nd.s_off = r.size;   // relative for now
      r.size += (sz + 31) / 32 * 32;
    }
    std::vector<Region*> placed;
    int64_t peak = 0;
    for (auto& kv : regions) {
      Region& r = kv.second;
      std::vector<int64_t> cand{0};
      for (Region* q : placed)
        if (q->start <= r.end && r.start <= q->end) cand.push_back(q->off + q->size);
      std::sort(cand.begin(), cand.end());
      for (int64_t off : cand) {
        bool ok = true;
        for (Region* q : placed)
          if (q->start <= r.end && r.start <= q->end && off < q->off + q->size && q->off < off + r.size) {
            ok = false;
            break;
          }
        if (ok) { r.off = off; break; }
      }
      placed.push_back(&r);
      peak = std::max(peak, r.off + r.size);
      for (int k : r.members) p.nodes[k].s_off += r.off;
    }
    (want64 ? p.s64_stride : p.s32_stride) = peak;
  }

  // maps: vid[nf-1] (gamma then boundary), pos0[nf], pos1[nf] (merge nodes)
  p.maps.clear();
  for (int k = 0; k < nn; ++k) {
    Node& nd = p.nodes[k];
    nd.map_off = (int64_t)p.maps.size();
    std::vector<int> rows(nd.gamma);
    rows.insert(rows.end(), nd.bnd.begin(), nd.bnd.end());
    p.maps.insert(p.maps.end(), rows.begin(), rows.end());
    if (nd.linv) {
      // the interior row coupled to each boundary row (-1: a corner, no interior neighbour)
      std::map<int, int> grow;
      for (int r = 0; r < nd.m; ++r) grow[nd.gamma[r]] = r;
      for (int v : nd.bnd) {
        const int vi = v % p.N, vj = v / p.N;
        int c = -1, hits = 0;
        const int nbr[4][2] = {{vi - 1, vj}, {vi + 1, vj}, {vi, vj - 1}, {vi, vj + 1}};
        for (const auto& q : nbr) {
          auto it = grow.find(q[1] * p.N + q[0]);
          if (it != grow.end()) { c = it->second; ++hits; }
        }
        if (hits > 1) return "internal: boundary vertex with two interior neighbours in a leaf";
        p.maps.push_back(c);
      }
    }
    if (!nd.leaf()) {
      for (int c = 0; c < 2; ++c) {
        const Node& ch = p.nodes[nd.child[c]];
        std::map<int, int> pos;
        for (int a = 0; a < ch.b; ++a) pos[ch.bnd[a]] = a;
        int covered = 0;
        for (int r = 0; r < nd.nf - 1; ++r) {
          auto it = pos.find(rows[r]);
          p.maps.push_back(it == pos.end() ? -1 : it->second);
          covered += it != pos.end();
        }
        p.maps.push_back(ch.b);   // right-hand-side row
        if (covered != ch.b) return "internal: son boundary not covered by the father front";
      }
    }
    if (p.maps.size() > (size_t)INT32_MAX) return "map table too large";
  }
  // up maps: for every non-root node, the father-front row of each of its Schur
  // rows (boundary unknowns, then the right-hand side)
  for (int k = 0; k < nn; ++k) {
    Node& nd = p.nodes[k];
    nd.up_off = (int64_t)p.maps.size();
    if (nd.parent < 0) continue;
    const Node& pa = p.nodes[nd.parent];
    std::map<int, int> prow;
    for (int r = 0; r < pa.m; ++r) prow[pa.gamma[r]] = r;
    for (int r = 0; r < pa.b; ++r) prow[pa.bnd[r]] = pa.m + r;
    for (int a = 0; a < nd.b; ++a) {
      auto it = prow.find(nd.bnd[a]);
      if (it == prow.end()) return "internal: son boundary vertex missing in the father front";
      p.maps.push_back(it->second);
    }
    p.maps.push_back(pa.nf - 1);
    if (p.maps.size() > (size_t)INT32_MAX) return "map table too large";
  }

  // concatenated node lists
  p.list_data.clear();
  p.lists.clear();
  auto add_list = [&](const std::vector<int>& v) {
    p.lists.push_back(make_list(p, v, p.list_data));
    return (int)p.lists.size() - 1;
  };
  p.step_lists.assign(p.height + 1, {0, 0, 0, 0, 0, 0, 0, 0});
  for (int hgt = 0; hgt <= p.height; ++hgt) {
    const Step& st = p.steps[hgt];
    p.step_lists[hgt] = {add_list(st.tiny64), add_list(st.small64), add_list(st.large64),
                         add_list(st.tiny32), add_list(st.small32), add_list(st.large32),
                         add_list(st.linv64), add_list(st.linv32)};
  }
  // right-hand-side sweep: every node (fused or not), by height, precision and format
  p.fwd_lists.assign(p.height + 1, {0, 0, 0, 0});
  {
    std::vector<std::vector<int>> l[4];
    for (auto& v : l) v.assign(p.height + 1, {});
    for (int k = 0; k < nn; ++k) {
      const Node& nd = p.nodes[k];
      l[(nd.linv ? 2 : 0) + (nd.fp64 ? 0 : 1)][nd.height].push_back(k);
    }
    for (int hgt = 0; hgt <= p.height; ++hgt)
      p.fwd_lists[hgt] = {add_list(l[0][hgt]), add_list(l[1][hgt]), add_list(l[2][hgt]), add_list(l[3][hgt])};
  }
  // mean functionals (mean plans): the observed nodes and their subtrees, by height,
  // precision and format; lambda^g offsets of the observed nodes
  p.func_lists.assign(p.height + 1, {0, 0, 0, 0});
  p.lam_off.assign(nn, -1);
  p.lam_stride = 0;
  if (p.obs_kind == HDD_OBS_MEANS) {
    std::vector<char> need(nn, 0);
    for (int k : p.obs_nodes) {
      need[k] = 1;
      if (p.lam_off[k] < 0) { p.lam_off[k] = (int32_t)p.lam_stride; p.lam_stride += p.nodes[k].b; }
    }
    for (int k = 1; k < nn; ++k)   // children have larger indices than their parent
      if (need[p.nodes[k].parent]) need[k] = 1;
    std::vector<std::vector<int>> l[4];
    for (auto& v : l) v.assign(p.height + 1, {});
    for (int k = 0; k < nn; ++k) {
      if (!need[k]) continue;
      const Node& nd = p.nodes[k];
      l[(nd.linv ? 2 : 0) + (nd.fp64 ? 0 : 1)][nd.height].push_back(k);
    }
    for (int hgt = 0; hgt <= p.height; ++hgt)
      p.func_lists[hgt] = {add_list(l[0][hgt]), add_list(l[1][hgt]), add_list(l[2][hgt]), add_list(l[3][hgt])};
  }
  // subdomain means: every node, by height
  {
    std::vector<std::vector<int>> l(p.height + 1);
    for (int k = 0; k < nn; ++k) l[p.nodes[k].height].push_back(k);
    p.height_lists.assign(p.height + 1, 0);
    for (int hgt = 0; hgt <= p.height; ++hgt) p.height_lists[hgt] = add_list(l[hgt]);
  }
  p.down_vis_lists.assign(p.depth + 1, {0, 0, 0});
  p.down_all_lists.assign(p.depth + 1, {0, 0, 0});
  for (int d = 0; d <= p.depth; ++d) {
    std::vector<int> vis[3], all[3];
    for (int k : p.down_all[d]) {
      const Node& nd = p.nodes[k];
      const int kind = nd.linv ? (nd.fp64 ? 1 : 2) : 0;
      all[kind].push_back(k);
      if (nd.visited) vis[kind].push_back(k);
    }
    p.down_vis_lists[d] = {add_list(vis[0]), add_list(vis[1]), add_list(vis[2])};
    p.down_all_lists[d] = {add_list(all[0]), add_list(all[1]), add_list(all[2])};
  }

  // device descriptors
  p.dev_nodes.resize(nn);
  for (int k = 0; k < nn; ++k) {
    const Node& nd = p.nodes[k];
    NodeDev& d = p.dev_nodes[k];
    d.m = nd.m; d.b = nd.b; d.nf = nd.nf; d.leaf = nd.linv ? 2 : (nd.leaf() ? 1 : 0);
    d.child0 = nd.child[0]; d.child1 = nd.child[1];
    d.x0 = nd.x0; d.y0 = nd.y0; d.x1 = nd.x1; d.y1 = nd.y1;
    d.map_off = (int32_t)nd.map_off;
    d.up_off = (int32_t)nd.up_off;
    d.fp64 = nd.fp64;
    d.y_off = (int32_t)nd.y_off;
    d.tc_off = nd.tc_off;
    d.inv_off = nd.inv_off;
    d.f_off = nd.f_off; d.s_off = nd.s_off;
  }

  // algorithmic flops (2 per multiply-add; leading terms):
  //   Cholesky m^3/3, TRSM (b+1) m^2/2, SYRK (b+1)(b+2)/2 m; descent b m + m^2/2
  p.flops_up = p.flops_down = 0.0;
  for (const Node& nd : p.nodes) {
    double m = nd.m, nb = nd.b + 1.0;
    p.flops_up += 2.0 * (m * m * m / 3.0 + nb * m * m / 2.0 + nb * (nb + 1.0) / 2.0 * m);
    if (nd.visited) p.flops_down += 2.0 * (nd.b * m + m * m / 2.0);
  }
  // algorithmic bytes per sample (see plan.h)
  p.by_tiny = p.by_small = p.by_large = p.by_fused = p.by_leaf = 0.0;
  p.by_fwd = p.by_desc_all = p.by_desc_vis = 0.0;
  auto esz = [](const Node& nd) { return nd.fp64 ? 8.0 : 4.0; };
  auto tri = [](double n) { return n * (n + 1.0) / 2.0; };
  for (const Node& nd : p.nodes) {
    const double E = esz(nd), m = nd.m, b = nd.b, nf = nd.nf;
    double in = 0.0, sons_cond = 0.0;
    if (nd.leaf()) {
      in = 2.0 * (nd.x1 - nd.x0) * (nd.y1 - nd.y0) * E;   // kappa of the leaf's triangles
    } else {
      for (int c = 0; c < 2; ++c) {
        const Node& ch = p.nodes[nd.child[c]];
        in += tri(ch.b + 1.0) * esz(ch);
        sons_cond += ch.b * esz(ch);
      }
    }
    if (nd.linv) {   // condensed leaf: G (packed) and the couplings instead of F
      const double g = tri(m) + b;
      p.by_leaf += in + (g + m + tri(b + 1.0)) * E;
      p.by_fwd += g * E + m * 8.0 + (m + b) * E;
      const double down = (g + m) * E + b * 8.0 + m * 8.0;
      p.by_desc_all += down;
      if (nd.visited) p.by_desc_vis += down;
      continue;
    }
    const double front = in + (nf * m + m + tri(b + 1.0)) * E;
    if (nd.fused) p.by_fused += front;
    else if (nd.nf <= kTinyMax) p.by_tiny += front;
    else if (nd.nf <= (nd.fp64 ? kSmallMax64 : kSmallMax32)) p.by_small += front;
    else p.by_large += front;
    const double fwd = (nf - 1.0) * m * E + m * 8.0 + sons_cond + (m + b) * E;
    const double down = (nf - 1.0) * m * E + m * E + b * 8.0 + m * 8.0;
    p.by_fwd += fwd;
    p.by_desc_all += down;
    if (nd.visited) p.by_desc_vis += down;
  }
  build_sweep(p, p.sweep_max_height);
  const double NN = (double)p.N * p.N;
  p.by_residual = 2.0 * p.n_t * 8.0 + 2.0 * NN * 8.0;   // kappa and u in, r out
  p.by_assemble = p.n_z * 8.0 + p.n_t * (p.precision == HDD_MIXED_FP32 ? 12.0 : 8.0);
  p.by_kl_basis = (double)p.n_t * p.n_z * 8.0;
  return "";
}

ListInfo make_list(const Plan& p, const std::vector<int>& v, std::vector<int32_t>& data) {
  ListInfo li;
  li.off = (int64_t)data.size();
  li.n = (int)v.size();
  for (int k : v) {
    data.push_back(k);
    const Node& nd = p.nodes[k];
    li.max_nf = std::max(li.max_nf, nd.nf);
    li.max_m = std::max(li.max_m, nd.m);
    li.max_b = std::max(li.max_b, nd.b);
    if (nd.leaf()) li.max_rect = std::max(li.max_rect, (nd.x1 - nd.x0 + 1) * (nd.y1 - nd.y0 + 1));
    const double m = nd.m, b = nd.b;
    li.fl_chol += 2.0 * m * m * m / 3.0;
    li.fl_trsm += 2.0 * (b + 1.0) * m * m / 2.0;
    li.fl_syrk += 2.0 * b * (b + 1.0) / 2.0 * m;
    li.fl_rhs += 2.0 * (b + 1.0) * m;
  }
  return li;
}

namespace {
size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
int64_t fac_block(const Node& nd) {   // padded factor block of a node (elements)
  const int64_t sz = nd.linv ? (int64_t)nd.m * (nd.m + 1) / 2 + nd.b : (int64_t)nd.nf * nd.m;
  return (sz + 31) / 32 * 32;
}
}  // namespace

void build_sweep(Plan& p, int max_height) {
  SweepSub out;
  const int nn = (int)p.nodes.size();
  auto eligible = [&](const Node& nd) {
    if (nd.linv) return nd.m <= kLeafInvMax && nd.b <= kLeafInvMaxB;
    return nd.m >= 1 && nd.m <= 32 && nd.nf - 1 <= 128;
  };
  for (int H = std::min(max_height, kSweepMaxHeight); H >= 1; --H) {
    SweepSub sw;
    sw.height = H;
    std::vector<int> roots;
    for (int k = 0; k < nn; ++k) {
      const Node& nd = p.nodes[k];
      if (nd.height <= H && (nd.parent < 0 || p.nodes[nd.parent].height > H)) roots.push_back(k);
    }
    bool ok = !roots.empty();
    const bool fp64 = ok && p.nodes[roots[0]].fp64;
    const size_t E = fp64 ? 8 : 4;
    std::vector<char> fused(nn, 0);
    for (size_t q = 0; q < roots.size() && ok; ++q) {
      const int r = roots[q];
      const Node& rt = p.nodes[r];
      // pre-order: father, son 0's subtree, son 1's subtree
      std::vector<int> order, todo{r};
      while (!todo.empty()) {
        const int k = todo.back();
        todo.pop_back();
        order.push_back(k);
        const Node& nd = p.nodes[k];
        if (!nd.leaf()) { todo.push_back(nd.child[1]); todo.push_back(nd.child[0]); }
      }
      const int w = rt.x1 - rt.x0 + 1, h = rt.y1 - rt.y0 + 1;
      int32_t desc[kSubInts] = {(int32_t)(sw.sched.size() / kSchedInts), (int32_t)order.size(),
                                (int32_t)sw.rec.size(), 0, rt.x0, rt.y0, w, h,
                                (int32_t)(rt.f_off & 0xffffffff), (int32_t)(rt.f_off >> 32), 0,
                                (int32_t)rt.y_off, 0, 0, 0, 0};
      const size_t rec0 = sw.rec.size();
      int64_t f_len = 0, y_len = 0;
      for (int k : order) {
        const Node& nd = p.nodes[k];
        if (!eligible(nd) || nd.fp64 != fp64 || (!nd.leaf() && nd.linv)) { ok = false; break; }
        fused[k] = 1;
        const int nr = nd.nf - 1;
        const int kind = nd.linv ? 2 : (nd.leaf() ? 1 : 0);
        const int b0 = nd.leaf() ? 0 : p.nodes[nd.child[0]].b, b1 = nd.leaf() ? 0 : p.nodes[nd.child[1]].b;
        // the depth-first layout puts the subtree's blocks one after the other
        if (nd.f_off != rt.f_off + f_len || nd.y_off != rt.y_off + y_len) { ok = false; break; }
        const int32_t ent[kSchedInts] = {k, kind | nd.m << 2 | nd.b << 8 | nd.nf << 20, (int32_t)(sw.rec.size() - rec0),
                                         (int32_t)nd.y_off, (int32_t)f_len, (int32_t)y_len, b0, b1};
        f_len += fac_block(nd);
        y_len += (nd.m + 3) / 4 * 4;
        sw.sched.insert(sw.sched.end(), ent, ent + kSchedInts);
        const int32_t* vid = p.maps.data() + nd.map_off;
        auto pad = [&]() { if (sw.rec.size() & 1) sw.rec.push_back(0); };
        for (int i = 0; i < nr; ++i) {
          const int x = vid[i] % p.N - rt.x0, y = vid[i] / p.N - rt.y0;
          if (x < 0 || x >= w || y < 0 || y >= h) { ok = false; break; }
          sw.rec.push_back((int16_t)(y * w + x));
        }
        pad();
        if (kind == 0) {   // positions in the sons' condensed right-hand sides
          for (int s = 0; s < 2; ++s) {
            const int32_t* pos = vid + nr + s * nd.nf;
            for (int i = 0; i < nr; ++i) sw.rec.push_back((int16_t)pos[i]);
            pad();
          }
        } else if (kind == 2) {   // interior row coupled to each boundary row
          for (int i = 0; i < nd.b; ++i) sw.rec.push_back((int16_t)vid[nr + i]);
          pad();
        }
      }
      if (!ok || (size_t)w * h > 32767 || f_len > (1 << 24)) { ok = false; break; }
      desc[3] = (int32_t)(sw.rec.size() - rec0);
      desc[10] = (int32_t)f_len;
      desc[12] = (int32_t)y_len;
      sw.f_elems = std::max(sw.f_elems, (int)f_len);
      sw.y_elems = std::max(sw.y_elems, (int)y_len);
      sw.subs.insert(sw.subs.end(), desc, desc + kSubInts);
      sw.max_nodes = std::max(sw.max_nodes, (int)order.size());
      sw.max_rec = std::max(sw.max_rec, desc[3]);
      sw.region_elems = std::max(sw.region_elems, w * h);
      // the sweep's stack of condensed right-hand sides (sons' on top of each other until
      // their father takes them), in the sweep's order: reversed pre-order
      int sp = 0, peak = 0;
      for (size_t i = order.size(); i-- > 1;) {
        const Node& nd = p.nodes[order[i]];
        if (!nd.leaf()) sp -= p.nodes[nd.child[0]].b + p.nodes[nd.child[1]].b;
        sp += nd.b;
        peak = std::max(peak, sp);
      }
      sw.stack_elems = std::max(sw.stack_elems, peak);
    }
    if (!ok) continue;
    sw.fp64 = fp64;
    sw.n_sub = (int)roots.size();
    const size_t shared = align16((size_t)sw.max_nodes * kSchedInts * 4) + align16((size_t)sw.max_rec * 2);
    const size_t fac = align16((size_t)sw.f_elems * E), yg = align16((size_t)sw.y_elems * E);
    const size_t region = align16((size_t)sw.region_elems * E), stack = align16((size_t)sw.stack_elems * E);
    sw.smem_desc = shared + kSubWarps * (fac + yg + region);
    sw.smem_fwd = shared + kSubWarps * (fac + region + stack);
    if (std::max(sw.smem_desc, sw.smem_fwd) > (size_t)kSubSmemCap) continue;
    // the descent's levels above the subtrees, by depth and kind
    sw.top_lists.assign(p.depth + 1, {0, 0, 0});
    for (int d = 0; d <= p.depth; ++d) {
      std::vector<int> all[3];
      for (int k : p.down_all[d]) {
        if (fused[k]) continue;
        const Node& nd = p.nodes[k];
        all[nd.linv ? (nd.fp64 ? 1 : 2) : 0].push_back(k);
      }
      for (int kind = 0; kind < 3; ++kind) {
        sw.top_infos.push_back(make_list(p, all[kind], sw.top_data));
        sw.top_lists[d][kind] = (int)sw.top_infos.size() - 1;
      }
    }
    out = std::move(sw);
    break;
  }
  p.sweep = std::move(out);
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Layout layout(const Plan& p, int batch) {
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
  const size_t B = (size_t)batch, NN = (size_t)p.N * p.N;
  L.status = take(B * 4);
  L.conv = take(B * 8);
  L.kappa = take(B * p.n_t * 8);
  if (p.precision == HDD_MIXED_FP32) L.kappa32 = take(B * p.n_t * 4);
  L.u = take(B * NN * 8);
  if (p.precision == HDD_MIXED_FP32) {
    L.r = take(B * NN * 8);
    L.du = take(B * NN * 8);
  }
  L.f64 = take(B * (size_t)p.f64_stride * 8);
  L.f32 = take(B * (size_t)p.f32_stride * 4);
  L.tc = take(B * (size_t)p.tc_stride);
  L.inv = take(B * (size_t)p.inv_stride);
  L.y64 = take(B * (size_t)p.y64_stride * 8);
  L.y32 = take(B * (size_t)p.y32_stride * 4);
  L.s64 = take(B * (size_t)p.s64_stride * 8);
  L.s32 = take(B * (size_t)p.s32_stride * 4);
  L.uobs = take(B * p.n_obs * 8);
  L.ll = take(B * 8);
  L.z = take(B * p.n_z * 8);
  L.y = take(B * p.n_obs * 8);
  if (p.obs_kind == HDD_OBS_MEANS) {
    L.fmu = take(B * p.nodes.size() * 8);
    L.lam = take(B * (size_t)p.lam_stride * 8);
    L.conv_u = take(B * (size_t)p.n_conv * 8);
    if (p.precision == HDD_MIXED_FP32 && p.ir_max_iter > 0) L.mfull = take(B * p.nodes.size() * 8);
  }
  L.total = off;
  return L;
}

}  // namespace hdd
