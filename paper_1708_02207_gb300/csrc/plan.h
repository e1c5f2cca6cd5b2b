// Internal plan of the HDD likelihood library: decomposition tree, fronts,
// index maps, launch schedule and workspace layout.  Host C++ only; the .cu
// files include it for the shared device descriptor.
#pragma once

#include <array>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hdd.h"

namespace hdd {

// Device-side node descriptor (88 bytes).  A node's front has nf = m + b + 1
// rows: m eliminated vertices (gamma, or a leaf's interior), b boundary unknowns,
// and one bordered right-hand-side row.  Per sample the front is stored as
//   F: nf x m column-major (ld nf)      -> L_gg (rows < m), L_Bg, y_g^T (last row)
//      (condensed leaves, leaf == 2: G = K_gg^-1 packed lower [m(m+1)/2], then the
//      boundary coupling weights [b]; y_g holds G b_g)
//   S: (b+1) x (b+1) column-major (ld b+1), lower triangle -> Schur complement and
//      condensed right-hand side (last row)
struct NodeDev {
  int32_t m, b, nf, leaf;
  int32_t child0, child1;
  int32_t x0, y0, x1, y1;   // closed rectangle (vertex indices)
  int32_t map_off;          // ints into the map table: vid[nf-1], then pos0[nf], pos1[nf]
  int32_t up_off;           // ints into the map table: father-front row of each Schur row [b+1]
  int32_t fp64;             // 1 if this node's factors are FP64 (mixed plans: top levels)
  int32_t y_off;            // elements into a sample's y arena of the node's type: y_g [m]
  int64_t f_off;            // elements into a sample's factor store of the node's type
  int64_t s_off;            // elements into a sample's Schur arena of the node's type
  int64_t tc_off;           // bytes into a sample's tensor-core staging arena, or -1
  int64_t inv_off;          // bytes into a sample's arena of inverted 32 x 32 diagonal blocks of L_gg, or -1
};
static_assert(sizeof(NodeDev) == 88, "NodeDev layout");

struct Node {
  int x0, x1, y0, y1;
  int depth = 0, height = 0;
  int parent = -1;
  int child[2] = {-1, -1};
  char split = 0;          // 'x': vertical line x = cut; 'y': horizontal line y = cut
  int cut = -1;
  std::vector<int> gamma;  // eliminated vertex ids, ordered
  std::vector<int> bnd;    // boundary unknowns, ascending id
  bool visited = false;
  bool fp64 = true;
  bool fused = false;      // eliminated inside a fused subtree
  bool linv = false;       // condensed leaf: stores K_gg^-1 and its boundary couplings instead of F
  int m = 0, b = 0, nf = 0;
  int64_t f_off = 0, s_off = 0, y_off = 0, tc_off = -1, inv_off = -1;
  int64_t map_off = 0;
  int64_t up_off = 0;
  bool leaf() const { return child[0] < 0; }
};

// A list of nodes launched together, with the maxima that size the launch.
struct ListInfo {
  int64_t off = 0;   // into the concatenated list table
  int n = 0;
  int max_nf = 0, max_m = 0, max_b = 0;
  int max_rect = 0;   // leaves: vertices of the largest closed rectangle
  double fl_chol = 0, fl_trsm = 0, fl_syrk = 0, fl_rhs = 0;   // algorithmic flops per sample
};

// One upsweep step: all nodes of one height, split by front size and precision.
struct Step {
  std::vector<int> tiny64, small64, large64, tiny32, small32, large32, linv64, linv32;
};

// Fused bottom subtrees of the right-hand-side sweep and of the full descent: one warp
// per (subtree, sample) keeps the vertex values of the subtree's rectangle in shared
// memory and copies the subtree's factor blocks (contiguous in the depth-first factor
// layout) into shared memory at once (k_sweep.cu).  A subtree is a node of height
// <= height whose father is higher, with all its descendants; every node in it has
// m <= 32 eliminated vertices and at most 128 front rows, or is a condensed leaf.
constexpr int kSweepMaxHeight = 6;        // largest subtree height allowed
constexpr int kSweepDefaultHeight = 2;    // a new plan's limit (fastest measured at 513^2 with 4 x 4-cell leaves)
constexpr int kSubInts = 16;              // ints per subtree descriptor
constexpr int kSchedInts = 8;             // ints per scheduled node
constexpr int kSubWarps = 8;              // warps (samples) per CTA
constexpr int kSubSmemCap = 75 * 1024;    // shared memory per CTA (three CTAs per SM)
struct SweepSub {
  int height = 0;            // 0: the sweeps run level by level
  bool fp64 = false;
  int n_sub = 0, max_nodes = 0, max_rec = 0;   // max_rec: int16 entries of one subtree's map records
  int region_elems = 0, stack_elems = 0;
  int f_elems = 0, y_elems = 0;                // largest factor and y_g ranges of a subtree
  size_t smem_desc = 0, smem_fwd = 0;          // bytes per CTA
  // per subtree: sched offset (nodes), node count, rec offset and length (int16 entries),
  // rectangle x0, y0, width, height (vertices), factor range start (lo, hi) and length,
  // y_g range start and length (elements of the subtree's precision), 3 unused
  std::vector<int32_t> subs;
  // per node, pre-order (root first): node, kind | m << 2 | b << 8 | nf << 20, rec offset
  // within the subtree's records, y_off, factor and y_g offsets within the subtree's
  // ranges, b of son 0, b of son 1
  std::vector<int32_t> sched;
  // per node: local index of each front row in the rectangle [nf-1]; then, for fathers,
  // the row's position in each son's condensed right-hand side [nf-1] x 2 (-1: none); for
  // condensed leaves, the interior row coupled to each boundary row [b]; each padded to even
  std::vector<int16_t> rec;
  // down_all_lists without the fused nodes (their own list table)
  std::vector<ListInfo> top_infos;
  std::vector<int32_t> top_data;
  std::vector<std::array<int, 3>> top_lists;
  int32_t* d_subs = nullptr;
  int32_t* d_sched = nullptr;
  int16_t* d_rec = nullptr;
  int32_t* d_top = nullptr;
};

struct Plan {
  // problem
  int N = 0, leaf = 0, n_z = 0, n_obs = 0, n_t = 0, device = -1;
  int obs_kind = HDD_OBS_VERTEX;
  // n_conv = obs.size(): the vertices whose corrections drive the refinement's
  // convergence test (vertex plans: the observations; mean plans: the boundary
  // unknowns of the observed nodes, or the root's interface)
  int n_conv = 0;
  std::vector<int32_t> obs_nodes;   // mean plans: the observed tree nodes
  int precision = HDD_FP64, ir_max_iter = 0, fp64_top_levels = 0, fuse_height = 0;
  double f = 1.0, sigma = 1.0, h = 0.0, ir_tol = 1e-10;
  std::vector<int32_t> obs;
  // bounded device waits: polls before a wait gives up, and the test hook that
  // withholds the copies of one (node, sample) (hdd_set_wait_bound)
  uint32_t wait_limit = 1u << 24;
  int stall_node = -1, stall_sample = -1;

  // tree
  std::vector<Node> nodes;
  std::vector<int32_t> owner;          // vertex id -> node that eliminates it (-1: Dirichlet)
  std::vector<Step> steps;             // by height, leaves first
  std::vector<std::vector<int>> down_visited, down_all;   // by depth, root first (condensed leaves excluded)
  std::vector<int32_t> maps;           // concatenated per-node maps
  std::vector<NodeDev> dev_nodes;
  int max_front = 0, max_front_small64 = 0, max_front_small32 = 0;
  int max_nf_large = 0, max_m_large = 0, max_b_large = 0;
  int n_leaves = 0, depth = 0, height = 0, n_visited = 0;

  // per-sample sizes (elements)
  int64_t f64_stride = 0, f32_stride = 0;   // factor stores
  int64_t y64_stride = 0, y32_stride = 0;   // y_g arenas (one entry per eliminated vertex)
  int64_t tc_stride = 0;                    // bytes: split TF32 tiles of one height step
  int64_t inv_stride = 0;                   // bytes: inverted diagonal blocks of one height step
  int64_t s64_stride = 0, s32_stride = 0;   // Schur arenas (lifetime-packed)
  double flops_up = 0.0, flops_down = 0.0;
  // algorithmic bytes per sample: each input read once and each output written
  // once (fronts: sons' lower Schur triangles or the leaf's kappa in; F, y_g and
  // the lower Schur triangle out)
  double by_tiny = 0.0, by_small = 0.0, by_large = 0.0, by_fused = 0.0;   // upsweep fronts by kernel class
  double by_leaf = 0.0;                                    // condensed leaves
  double by_fwd = 0.0;                                     // one right-hand-side sweep
  double by_desc_all = 0.0, by_desc_vis = 0.0;             // full and pruned descents
  double by_residual = 0.0, by_assemble = 0.0;             // FP64 residual; kappa written
  double by_kl_basis = 0.0;                                // Phi, read once per batch

  // fused bottom subtrees, per precision (0: FP64, 1: FP32)
  struct Fusion {
    int height = 0;                 // subtree height (0: no fusion)
    std::vector<int32_t> roots;     // 12 ints per subtree
    std::vector<int32_t> nodes;     // node lists
    int sbuf_elems = 0, front_elems = 0;
    size_t smem_bytes = 0;
    int32_t* d_roots = nullptr;
    int32_t* d_nodes = nullptr;
  } fusion[2];
  std::vector<int32_t> fuse_soff;   // per node
  int32_t* d_fuse_soff = nullptr;

  // fused bottom subtrees of the sweeps (hdd_set_sweep_fusion)
  SweepSub sweep;
  int sweep_max_height = kSweepDefaultHeight;

  // node lists concatenated (host copy of d_lists) and their descriptors
  std::vector<int32_t> list_data;
  std::vector<ListInfo> lists;
  // [height][tiny64, small64, large64, tiny32, small32, large32, linv64, linv32]
  std::vector<std::array<int, 8>> step_lists;
  // [depth][fp64 and fp32 fronts, condensed leaves (fp64), condensed leaves (fp32)]
  std::vector<std::array<int, 3>> down_vis_lists, down_all_lists;
  // [height][fp64, fp32, condensed fp64, condensed fp32]: right-hand-side sweep
  std::vector<std::array<int, 4>> fwd_lists;
  std::vector<int> height_lists;   // per height: every node (subdomain means)
  // mean plans: per height [fp64, fp32, condensed fp64, condensed fp32] nodes whose mean
  // functional is needed (the observed nodes and their subtrees), and per node the
  // offset of its functional lambda^g in the workspace's observation block (-1: none)
  std::vector<std::array<int, 4>> func_lists;
  std::vector<int32_t> lam_off;
  int64_t lam_stride = 0;          // sum of b over the observed nodes
  int32_t* d_lam_off = nullptr;
  int32_t* d_obs_nodes = nullptr;

  // device copies
  double* d_phi = nullptr;
  float* d_phi_hi = nullptr;   // mixed plans: Phi as FP32 hi + lo pairs
  float* d_phi_lo = nullptr;
  NodeDev* d_nodes = nullptr;
  int32_t* d_maps = nullptr;
  int32_t* d_lists = nullptr;
  int32_t* d_obs = nullptr;
};

// Fronts of at most kTinyMax rows run one per warp in registers; up to the
// kSmallMax limits one per CTA in shared memory; larger ones in global memory.
constexpr int kTinyMax = 32;
// Largest height of a fused bottom subtree allowed by the kernel.
constexpr int kFuseMaxHeight = 6;
// Tensor-core SYRK staging: 128-row tiles x 8-column chunks, hi and lo parts of
// 4 KiB each (TF32 values in the 8-row x 16-byte core-matrix layout).
constexpr int kTcTile = 128, kTcChunk = 8;
constexpr int64_t kTcBlockBytes = (int64_t)kTcTile * kTcChunk * 4;
constexpr int kSmallMax64 = 160;   // 160^2 * 8 B = 200 KiB
constexpr int kSmallMax32 = 128;   // 128 * 132 * 4 B = 66 KiB (larger FP32 fronts: tensor-core path)
// Condensed leaves: leaves with 1..kLeafInvMax interior vertices and at most
// kLeafInvMaxB boundary unknowns store, per sample, G = K_gg^-1 (packed lower,
// column-major) followed by the coupling weight of each boundary row (on this
// mesh every boundary vertex of a rectangle has at most one interior neighbour).
constexpr int kLeafInvMax = 16;
constexpr int kLeafInvMaxB = 63;

// Build the host plan; returns an empty string on success, else an error text.
std::string build_plan(const hdd_plan_desc& d, Plan& p);
// The fused sweep subtrees of a built plan for subtree heights up to max_height (0: none);
// host tables only (the caller uploads them).
void build_sweep(Plan& p, int max_height);
// A node list's descriptor (sizes and algorithmic flops), its nodes appended to data.
ListInfo make_list(const Plan& p, const std::vector<int>& v, std::vector<int32_t>& data);

// Workspace layout for a batch (byte offsets, 256-byte aligned).
struct Layout {
  size_t status = 0, kappa = 0, kappa32 = 0;
  size_t u = 0, r = 0, du = 0;        // FP64 vertex vectors [batch x N^2]
  size_t f64 = 0, f32 = 0, s64 = 0, s32 = 0, y64 = 0, y32 = 0, tc = 0, inv = 0;
  size_t uobs = 0, ll = 0, z = 0, y = 0, conv = 0;
  // mean plans: mu^f of every node [batch x n_nodes], lambda^g of the observed nodes
  // [batch x lam_stride], the corrected vertices of the convergence test
  // [batch x n_conv], and (mixed plans with refinement) the means of the refined
  // iterate [batch x n_nodes]
  size_t fmu = 0, lam = 0, conv_u = 0, mfull = 0;
  size_t total = 0;
};
Layout layout(const Plan& p, int batch);

}  // namespace hdd

// The opaque plan handle of the C ABI.
struct hdd_plan_s {
  hdd::Plan p;
  void* prof = nullptr;   // per-kernel timing state (api.cu), or nullptr
};
