// Host check of the fused sweep subtrees' tables (plan.cpp, build_sweep) against the
// index arithmetic of k_descent_sub / k_forward_sub (k_sweep.cu), over real plans:
//   * every node of height <= the subtree height lies in exactly one subtree;
//   * the schedule repeats the node's sizes, and each node's factor and y_g blocks lie
//     at the given offsets inside its subtree's contiguous, 16-byte aligned ranges,
//     which lie inside the per-sample stores;
//   * the map records stay inside their subtree's block: rectangle indices inside the
//     rectangle, positions inside the sons' condensed loads, couplings inside gamma;
//   * the descent reads a boundary value only after it is known (the root's border,
//     gathered, or an ancestor's gamma), writes every gamma once, and covers the
//     rectangle's interior;
//   * the sweep finds son 0's condensed load on top of son 1's when their father
//     takes them, and the stack never exceeds its size;
//   * the shared memory layout adds up to the launch's size.
// Usage: sweep_tables_check N leaf precision fp64_top_levels max_height; prints the
// height in use and exits 0, or prints the failed check and exits 1.
#include <cstdio>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include "plan.h"

using namespace hdd;

#define CHECK(c, ...)                                   \
  do {                                                  \
    if (!(c)) {                                         \
      std::printf("FAIL line %d: ", __LINE__);          \
      std::printf(__VA_ARGS__);                         \
      std::printf("\n");                                \
      std::exit(1);                                     \
    }                                                   \
  } while (0)

namespace {

struct Entry {
  int node, kind, m, b, nf, rec, y_off, f_rel, y_rel, b0, b1;
};

Entry decode(const int32_t* e) {
  Entry q;
  q.node = e[0];
  q.kind = e[1] & 3;
  q.m = (e[1] >> 2) & 63;
  q.b = (e[1] >> 8) & 4095;
  q.nf = (e[1] >> 20) & 2047;
  q.rec = e[2];
  q.y_off = e[3];
  q.f_rel = e[4];
  q.y_rel = e[5];
  q.b0 = e[6];
  q.b1 = e[7];
  return q;
}

size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
int pad2(int n) { return (n + 1) & ~1; }

}  // namespace

int main(int argc, char** argv) {
  CHECK(argc == 6, "usage: N leaf precision fp64_top_levels max_height");
  const int N = std::atoi(argv[1]), leaf = std::atoi(argv[2]);
  hdd_plan_desc d{};
  d.N = N;
  d.leaf = leaf;
  d.n_z = 1;
  d.f = 1.0;
  d.n_obs = 1;
  int32_t obs = (N / 2) * N + N / 2;
  d.obs_vertex = &obs;
  d.sigma = 1.0;
  d.precision = std::atoi(argv[3]);
  d.fp64_top_levels = std::atoi(argv[4]);
  d.ir_tol = 1e-8;
  d.device = -1;
  Plan p;
  p.sweep_max_height = std::atoi(argv[5]);
  const std::string err = build_plan(d, p);
  CHECK(err.empty(), "build_plan: %s", err.c_str());
  const SweepSub& sw = p.sweep;
  if (sw.height == 0) {
    std::printf("height 0\n");
    return 0;
  }
  const size_t E = sw.fp64 ? 8 : 4;
  const size_t shared = al16((size_t)sw.max_nodes * kSchedInts * 4) + al16((size_t)sw.max_rec * 2);
  const size_t fac = al16(sw.f_elems * E), yg = al16(sw.y_elems * E);
  const size_t region = al16(sw.region_elems * E), stack = al16(sw.stack_elems * E);
  CHECK(shared + kSubWarps * (fac + yg + region) == sw.smem_desc, "descent shared memory");
  CHECK(shared + kSubWarps * (fac + region + stack) == sw.smem_fwd, "sweep shared memory");
  CHECK(sw.smem_desc <= (size_t)kSubSmemCap && sw.smem_fwd <= (size_t)kSubSmemCap, "shared memory cap");
  CHECK((int)sw.subs.size() == sw.n_sub * kSubInts, "descriptor count");
  std::vector<int> covered(p.nodes.size(), 0);
  for (int t = 0; t < sw.n_sub; ++t) {
    const int32_t* D = &sw.subs[(size_t)t * kSubInts];
    const int n = D[1], x0 = D[4], y0 = D[5], w = D[6], h = D[7];
    const int64_t froot = (int64_t)(uint32_t)D[8] | ((int64_t)D[9] << 32);
    CHECK(n >= 1 && n <= sw.max_nodes && D[3] <= sw.max_rec && D[2] % 2 == 0 && D[3] % 2 == 0, "subtree sizes");
    CHECK(w * h <= sw.region_elems, "rectangle size");
    CHECK((size_t)(D[0] + n) * kSchedInts <= sw.sched.size() && (size_t)(D[2] + D[3]) <= sw.rec.size(), "table ranges");
    CHECK((froot * (int64_t)E) % 16 == 0 && ((int64_t)D[11] * (int64_t)E) % 16 == 0, "range alignment");
    CHECK(D[10] <= sw.f_elems && D[12] <= sw.y_elems, "range lengths");
    const int64_t fstride = sw.fp64 ? p.f64_stride : p.f32_stride, ystride = sw.fp64 ? p.y64_stride : p.y32_stride;
    CHECK(froot + (int64_t)al16(D[10] * E) / (int64_t)E <= fstride, "factor range in the store");
    CHECK(D[11] + (int64_t)al16(D[12] * E) / (int64_t)E <= ystride, "y_g range in the store");
    const int16_t* rec = &sw.rec[D[2]];
    std::vector<Entry> q(n);
    for (int k = 0; k < n; ++k) q[k] = decode(&sw.sched[(size_t)(D[0] + k) * kSchedInts]);
    for (int k = 0; k < n; ++k) {
      const Node& nd = p.nodes[q[k].node];
      CHECK(q[k].m == nd.m && q[k].b == nd.b && q[k].nf == nd.nf && q[k].y_off == nd.y_off, "schedule sizes");
      CHECK(q[k].kind == (nd.linv ? 2 : nd.leaf() ? 1 : 0), "node kind");
      CHECK(nd.fp64 == sw.fp64 && nd.height <= sw.height, "precision and height");
      CHECK(covered[q[k].node]++ == 0, "node %d in two subtrees", q[k].node);
      const int64_t blk = q[k].kind == 2 ? (int64_t)q[k].m * (q[k].m + 1) / 2 + q[k].b : (int64_t)q[k].nf * q[k].m;
      CHECK(nd.f_off == froot + q[k].f_rel && q[k].f_rel >= 0 && q[k].f_rel + blk <= D[10], "factor block");
      CHECK(nd.y_off == D[11] + q[k].y_rel && q[k].y_rel >= 0 && q[k].y_rel + q[k].m <= D[12], "y_g block");
      if (q[k].kind == 2)
        CHECK(q[k].m <= kLeafInvMax && q[k].b <= kLeafInvMaxB, "condensed leaf size");
      else
        CHECK(q[k].m <= 32 && q[k].nf - 1 <= 128, "front size");
      const int nr = q[k].nf - 1;
      const int len = pad2(nr) + (q[k].kind == 0 ? 2 * pad2(nr) : q[k].kind == 2 ? pad2(q[k].b) : 0);
      CHECK(q[k].rec >= 0 && q[k].rec + len <= D[3], "record inside the subtree's block");
      for (int r = 0; r < nr; ++r) CHECK(rec[q[k].rec + r] >= 0 && rec[q[k].rec + r] < w * h, "rectangle index");
      if (!nd.leaf())
        CHECK(q[k].b0 == p.nodes[nd.child[0]].b && q[k].b1 == p.nodes[nd.child[1]].b, "sons' sizes");
      if (q[k].kind == 0)
        for (int r = 0; r < nr; ++r) {
          const int a = rec[q[k].rec + pad2(nr) + r], c = rec[q[k].rec + 2 * pad2(nr) + r];
          CHECK(a >= -1 && a < q[k].b0 && c >= -1 && c < q[k].b1, "son position");
        }
      if (q[k].kind == 2)
        for (int i = 0; i < q[k].b; ++i) {
          const int ci = rec[q[k].rec + pad2(nr) + i];
          CHECK(ci >= -1 && ci < q[k].m, "coupling row");
        }
    }
    // descent: every boundary value is known before it is read
    std::vector<char> known((size_t)w * h, 0);
    {
      const Node& rt = p.nodes[q[0].node];
      const int32_t* vid = p.maps.data() + rt.map_off;
      for (int i = 0; i < rt.b; ++i) {
        const int v = vid[rt.m + i], xx = v % N - x0, yy = v / N - y0;
        CHECK(rec[q[0].rec + rt.m + i] == yy * w + xx, "root boundary index");
        known[(size_t)yy * w + xx] = 1;
      }
    }
    for (int k = 0; k < n; ++k) {
      const int nr = q[k].nf - 1;
      for (int r = q[k].m; r < nr; ++r) CHECK(known[rec[q[k].rec + r]], "boundary value read before it is known");
      for (int r = 0; r < q[k].m; ++r) {
        const int l = rec[q[k].rec + r];
        CHECK(!known[l], "gamma written twice");
        CHECK(l % w >= 1 && l % w < w - 1 && l / w >= 1 && l / w < h - 1, "gamma inside the rectangle");
        known[l] = 1;
      }
    }
    for (int yy = 1; yy < h - 1; ++yy)
      for (int xx = 1; xx < w - 1; ++xx) CHECK(known[(size_t)yy * w + xx], "interior vertex not computed");
    // sweep: stack order and size (reversed pre-order, the root writes to global memory)
    std::vector<int> stk;
    int sp = 0;
    for (int k = n - 1; k >= 1; --k) {
      const Node& nd = p.nodes[q[k].node];
      if (q[k].kind == 0) {
        CHECK(stk.size() >= 2 && stk.back() == nd.child[0] && stk[stk.size() - 2] == nd.child[1], "stack order");
        sp -= q[k].b0 + q[k].b1;
        CHECK(sp >= 0, "stack underflow");
        stk.pop_back();
        stk.pop_back();
      }
      CHECK(sp + q[k].b <= sw.stack_elems, "stack overflow");
      sp += q[k].b;
      stk.push_back(q[k].node);
    }
    if (q[0].kind == 0) CHECK(stk.size() == 2 && sp == q[0].b0 + q[0].b1, "the root's sons at the end");
  }
  for (size_t k = 0; k < p.nodes.size(); ++k)
    CHECK((p.nodes[k].height <= sw.height) == (covered[k] == 1), "coverage of node %zu", k);
  std::printf("height %d subtrees %d\n", sw.height, sw.n_sub);
  return 0;
}
