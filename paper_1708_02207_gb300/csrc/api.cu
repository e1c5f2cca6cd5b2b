// C ABI of libhdd.so: plan management, workspace layout and the per-call launch
// schedule of the HDD likelihood path.  No exceptions cross this boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace hdd {
cudaError_t configure_front_kernels();
cudaError_t configure_solve_kernels();
cudaError_t configure_refine_kernels();
cudaError_t configure_warp_kernels();
cudaError_t configure_tc_kernels();
cudaError_t configure_fused_kernels();
cudaError_t configure_group_kernels();
cudaError_t configure_leaf_kernels();
cudaError_t configure_func_kernels();
cudaError_t configure_data_kernels();
cudaError_t configure_sweep_kernels();
}  // namespace hdd

namespace {

thread_local std::string g_err;

// Sweeps over nodes whose interface has at least this many vertices use one CTA
// per (node, sample) with blocked substitution; smaller nodes one warp each.
constexpr int kSweepCtaMinM = 16;
// right-hand-side sweeps of lists whose fronts have 16..32 eliminated vertices and at
// most 256 rows: one warp per (node, sample) with the rows in registers (measured faster
// there than the CTA kernel; below 16 the staged warp kernel stays faster, and for the
// descent the CTA kernel)
bool mid_list(const hdd::ListInfo& li) {
  return li.max_m >= kSweepCtaMinM && li.max_m <= 32 && li.max_nf - 1 <= hdd::kMidMaxRows;
}

hdd_status fail_cuda(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return HDD_ECUDA;
}

hdd_status fail_inval(const std::string& msg) {
  g_err = msg;
  return HDD_EINVAL;
}

}  // namespace

namespace hdd {
// Error text for hdd_last_error() from the other translation units of the library.
hdd_status set_error(hdd_status status, const std::string& msg) {
  g_err = msg;
  return status;
}

// The sizes and algorithmic flops of one node list on a launch's arguments
// (flops per sample of the list, times `scale`).
void set_list(StepArgs& a, const ListInfo& li, double scale) {
  a.nlist = li.n;
  a.max_nf = li.max_nf;
  a.max_m = li.max_m;
  a.max_b = li.max_b;
  a.max_rect = li.max_rect;
  a.fl_chol = li.fl_chol * scale;
  a.fl_trsm = li.fl_trsm * scale;
  a.fl_syrk = li.fl_syrk * scale;
  a.fl_rhs = li.fl_rhs * scale;
}

// One upsweep launch (or launch sequence, for the large fronts) over a node list of
// one height and one class: 0-2 FP64 fronts of up to 32 rows / in shared memory /
// in global memory, 3-5 the same in FP32, 6-7 condensed leaves (FP64, FP32).
cudaError_t launch_step(int kind, StepArgs& a, cudaStream_t st) {
  switch (kind) {
    case 0: return launch_front_group<double>(a, kProfFrontWarp, st);
    case 1: return launch_front_group<double>(a, kProfFrontSmall, st);
    case 2: return launch_front_large<double>(a, st);
    case 3: return launch_front_group<float>(a, kProfFrontWarp, st);
    case 4: return launch_front_group<float>(a, kProfFrontSmall, st);
    case 5: return launch_front_large<float>(a, st);
    case 6: return launch_leaf_front<double>(a, st);
    default: return launch_leaf_front<float>(a, st);
  }
}

// Launches of one upsweep list of the given class (the large fronts take a sequence).
int step_launches(int kind, const ListInfo& li) {
  if (li.n == 0) return 0;
  if (kind == 2) return li.max_m <= 32 ? 3 : 4;   // fill, POTRF+TRSM or POTRF, TRSM, SYRK
  if (kind == 5) return (li.max_m <= 64 ? 3 : 4) + (li.max_b > 0 ? 1 : 0);   // + bordered row
  return 1;
}
}  // namespace hdd

namespace {

// Makes the plan's device current for the duration of a call.
struct DeviceScope {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceScope(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

std::mutex g_cfg_mutex;
bool g_configured[64] = {};

cudaError_t configure_device(int dev) {
  std::lock_guard<std::mutex> lk(g_cfg_mutex);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (g_configured[dev]) return cudaSuccess;
  cudaError_t e = hdd::configure_front_kernels();
  if (e == cudaSuccess) e = hdd::configure_solve_kernels();
  if (e == cudaSuccess) e = hdd::configure_refine_kernels();
  if (e == cudaSuccess) e = hdd::configure_warp_kernels();
  if (e == cudaSuccess) e = hdd::configure_tc_kernels();
  if (e == cudaSuccess) e = hdd::configure_fused_kernels();
  if (e == cudaSuccess) e = hdd::configure_group_kernels();
  if (e == cudaSuccess) e = hdd::configure_leaf_kernels();
  if (e == cudaSuccess) e = hdd::configure_func_kernels();
  if (e == cudaSuccess) e = hdd::configure_data_kernels();
  if (e == cudaSuccess) e = hdd::configure_sweep_kernels();
  if (e == cudaSuccess) g_configured[dev] = true;
  return e;
}

void free_sweep(hdd::SweepSub& sw) {
  cudaFree(sw.d_subs);
  cudaFree(sw.d_sched);
  cudaFree(sw.d_rec);
  cudaFree(sw.d_top);
  sw.d_subs = sw.d_sched = sw.d_top = nullptr;
  sw.d_rec = nullptr;
}

void free_device(hdd::Plan& p) {
  cudaFree(p.d_phi);
  cudaFree(p.d_phi_hi);
  cudaFree(p.d_phi_lo);
  p.d_phi_hi = nullptr; p.d_phi_lo = nullptr;
  cudaFree(p.d_nodes);
  cudaFree(p.d_maps);
  cudaFree(p.d_lists);
  cudaFree(p.d_obs);
  for (auto& fu : p.fusion) {
    cudaFree(fu.d_roots);
    cudaFree(fu.d_nodes);
    fu.d_roots = fu.d_nodes = nullptr;
  }
  cudaFree(p.d_fuse_soff);
  p.d_fuse_soff = nullptr;
  free_sweep(p.sweep);
  cudaFree(p.d_lam_off);
  cudaFree(p.d_obs_nodes);
  p.d_lam_off = p.d_obs_nodes = nullptr;
  p.d_phi = nullptr; p.d_nodes = nullptr; p.d_maps = nullptr; p.d_lists = nullptr; p.d_obs = nullptr;
}

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  cudaError_t e = cudaMalloc((void**)dst, (n ? n : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t upload_sweep(hdd::SweepSub& sw) {
  if (sw.height == 0) return cudaSuccess;
  cudaError_t e = upload(&sw.d_subs, sw.subs.data(), sw.subs.size());
  if (e == cudaSuccess) e = upload(&sw.d_sched, sw.sched.data(), sw.sched.size());
  if (e == cudaSuccess) e = upload(&sw.d_rec, sw.rec.data(), sw.rec.size());
  if (e == cudaSuccess) e = upload(&sw.d_top, sw.top_data.data(), sw.top_data.size());
  return e;
}

hdd::Arenas arenas(const hdd::Plan& p, const hdd::Layout& L, void* ws) {
  char* w = static_cast<char*>(ws);
  hdd::Arenas A;
  A.f64 = reinterpret_cast<double*>(w + L.f64);
  A.f64_stride = p.f64_stride;
  A.f32 = reinterpret_cast<float*>(w + L.f32);
  A.f32_stride = p.f32_stride;
  A.s64 = reinterpret_cast<double*>(w + L.s64);
  A.s64_stride = p.s64_stride;
  A.s32 = reinterpret_cast<float*>(w + L.s32);
  A.s32_stride = p.s32_stride;
  A.y64 = reinterpret_cast<double*>(w + L.y64);
  A.y64_stride = p.y64_stride;
  A.y32 = reinterpret_cast<float*>(w + L.y32);
  A.y32_stride = p.y32_stride;
  A.tc = reinterpret_cast<unsigned char*>(w + L.tc);
  A.tc_stride = p.tc_stride;
  A.inv = reinterpret_cast<unsigned char*>(w + L.inv);
  A.inv_stride = p.inv_stride;
  return A;
}

}  // namespace

namespace hdd {
PlanDev plan_part(const Plan& p, int batch, void* ws) {
  const Layout L = layout(p, batch);
  char* w = static_cast<char*>(ws);
  PlanDev d{};
  d.arenas = arenas(p, L, ws);
  d.kappa = reinterpret_cast<const double*>(w + L.kappa);
  d.kappa32 = L.kappa32 ? reinterpret_cast<const float*>(w + L.kappa32) : nullptr;
  d.kap_stride = p.n_t;
  d.status = reinterpret_cast<int32_t*>(w + L.status);
  d.rhs = Rhs{nullptr, 0, p.h * p.h * p.f};
  d.N = p.N;
  d.batch = batch;
  return d;
}
}  // namespace hdd

namespace {

hdd_status check_call(hdd_plan_t plan, int32_t batch, void* ws) {
  if (!plan) return fail_inval("plan is NULL");
  if (plan->p.device < 0) {
    g_err = "host-only plan";
    return HDD_ESTATE;
  }
  if (batch < 1 || batch > 65535) return fail_inval("batch must be in 1..65535");
  if (!ws) return fail_inval("workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return fail_inval("workspace must be 256-byte aligned");
  return HDD_OK;
}

hdd::Profiler* profiler(hdd_plan_t plan) {
  hdd::Profiler* pr = static_cast<hdd::Profiler*>(plan->prof);
  return (pr && pr->on) ? pr : nullptr;
}

struct ProfScope {
  hdd::Profiler* pr;
  cudaStream_t st;
  ProfScope(hdd::Profiler* p, int fam, double fl, cudaStream_t s) : pr(p), st(s) {
    if (pr) pr->begin(fam, fl, st);
  }
  ~ProfScope() {
    if (pr) pr->end(st);
  }
};

// One pass of "Leaves to Root" over all heights with the given right-hand side.
cudaError_t run_upsweep(const hdd::Plan& p, int batch, void* ws, const hdd::Rhs& rhs, cudaStream_t st,
                        hdd::Profiler* prof) {
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(ws);
  hdd::StepArgs a{};
  a.nodes = p.d_nodes;
  a.maps = p.d_maps;
  a.batch = batch;
  a.N = p.N;
  a.kappa = reinterpret_cast<const double*>(w + L.kappa);
  a.kappa32 = L.kappa32 ? reinterpret_cast<const float*>(w + L.kappa32) : nullptr;
  a.kap_stride = p.n_t;
  a.rhs = rhs;
  a.arenas = arenas(p, L, ws);
  a.status = reinterpret_cast<int32_t*>(w + L.status);
  a.prof = prof;
  a.wait_limit = p.wait_limit;
  a.stall_node = p.stall_node;
  a.stall_sample = p.stall_sample;
  // fused bottom subtrees first (their roots' Schur blocks feed the regular steps)
  for (int prec = 0; prec < 2; ++prec) {
    const hdd::Plan::Fusion& fu = p.fusion[prec];
    if (fu.height == 0) continue;
    hdd::FuseArgs fa;
    fa.a = a;
    fa.roots = fu.d_roots;
    fa.fused = fu.d_nodes;
    fa.fuse_soff = p.d_fuse_soff;
    fa.sbuf_elems = fu.sbuf_elems;
    fa.front_elems = fu.front_elems;
    const int nroots = (int)fu.roots.size() / 12;
    double fl = 0.0;
    for (int q : fu.nodes) {
      const double m = p.nodes[q].m, b = p.nodes[q].b;
      fl += 2.0 * (m * m * m / 3.0 + (b + 1.0) * m * m / 2.0 + (b + 1.0) * (b + 2.0) / 2.0 * m);
    }
    ProfScope ps(prof, hdd::kProfFused, fl * batch, st);
    cudaError_t e = prec == 0 ? hdd::launch_subtree<double>(fa, nroots, fu.smem_bytes, st)
                              : hdd::launch_subtree<float>(fa, nroots, fu.smem_bytes, st);
    if (e != cudaSuccess) return e;
  }
  for (int h = 0; h <= p.height; ++h) {
    for (int kind = 0; kind < 8; ++kind) {
      const hdd::ListInfo& li = p.lists[p.step_lists[h][kind]];
      if (li.n == 0) continue;
      a.list = p.d_lists + li.off;
      hdd::set_list(a, li, batch);
      cudaError_t e = hdd::launch_step(kind, a, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// The sweeps' fused bottom subtrees of a plan for one batch.
hdd::SubArgs sub_args(const hdd::Plan& p, int batch, const hdd::Arenas& A, bool descent) {
  const hdd::SweepSub& sw = p.sweep;
  const size_t E = sw.fp64 ? 8 : 4;
  auto al16 = [](size_t x) { return (int)((x + 15) & ~(size_t)15); };
  hdd::SubArgs g{};
  g.nodes = p.d_nodes;
  g.maps = p.d_maps;
  g.subs = sw.d_subs;
  g.sched = sw.d_sched;
  g.rec = sw.d_rec;
  g.A = A;
  g.N = p.N;
  g.batch = batch;
  g.fac_bytes = al16((size_t)sw.f_elems * E);
  g.y_bytes = descent ? al16((size_t)sw.y_elems * E) : 0;
  g.region_bytes = al16((size_t)sw.region_elems * E);
  g.stack_bytes = descent ? 0 : al16((size_t)sw.stack_elems * E);
  g.warp_bytes = g.fac_bytes + g.y_bytes + g.region_bytes + g.stack_bytes;
  g.sched_bytes = al16((size_t)sw.max_nodes * hdd::kSchedInts * 4);
  g.rec_bytes = al16((size_t)sw.max_rec * 2);
  return g;
}

// "Root to Leaves" over per-depth lists (indices into `infos`; nodes in `data` on the
// host and at d_base on the device, at each list's offset).
cudaError_t descent_levels(const hdd::Plan& p, int batch, const hdd::Arenas& A,
                           const std::vector<std::array<int, 3>>& per_depth, const std::vector<hdd::ListInfo>& infos,
                           const std::vector<int32_t>& data, const int32_t* d_base, double* u, int64_t u_stride,
                           cudaStream_t st, hdd::Profiler* prof) {
  for (int d = 0; d < (int)per_depth.size(); ++d) {
    for (int kind = 1; kind < 3; ++kind) {   // condensed leaves of this depth
      const hdd::ListInfo& ll = infos[per_depth[d][kind]];
      if (ll.n == 0) continue;
      ProfScope ps(prof, hdd::kProfDescent, 0.0, st);
      cudaError_t e = kind == 1 ? hdd::launch_leaf_descent<double>(p.d_nodes, p.d_maps, d_base + ll.off, ll.n,
                                                                   batch, A, u, u_stride, st)
                                : hdd::launch_leaf_descent<float>(p.d_nodes, p.d_maps, d_base + ll.off, ll.n,
                                                                  batch, A, u, u_stride, st);
      if (e != cudaSuccess) return e;
    }
    const hdd::ListInfo& li = infos[per_depth[d][0]];
    if (li.n == 0) continue;
    // the lists hold one precision per depth in the plans built here
    const bool fp64 = p.nodes[data[li.off]].fp64;
    // nodes with long interfaces: one CTA per (node, sample), blocked back substitution;
    // otherwise one warp per (node, sample)
    const bool cta = li.max_m >= kSweepCtaMinM;
    const int32_t* list = d_base + li.off;
    ProfScope ps(prof, hdd::kProfDescent, 0.0, st);
    cudaError_t e;
    if (li.max_nf <= hdd::kTinyMax)
      e = fp64 ? hdd::launch_descent_tiny<double>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, st)
               : hdd::launch_descent_tiny<float>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, st);
    else if (cta)
      e = fp64 ? hdd::launch_descent<double>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, li.max_b,
                                             li.max_m, st)
               : hdd::launch_descent<float>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, li.max_b,
                                            li.max_m, st);
    else
      e = fp64 ? hdd::launch_descent_warp<double>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, li.max_nf,
                                                  li.max_m, st)
               : hdd::launch_descent_warp<float>(p.d_nodes, p.d_maps, list, li.n, batch, A, u, u_stride, li.max_nf,
                                                 li.max_m, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// "Root to Leaves" over the given per-depth lists, writing u (FP64).  The full descent
// of a plan with fused sweep subtrees runs the levels above them, then the subtrees.
cudaError_t run_descent(const hdd::Plan& p, int batch, void* ws, const std::vector<std::array<int, 3>>& per_depth,
                        double* u, int64_t u_stride, cudaStream_t st, hdd::Profiler* prof) {
  const hdd::Layout L = hdd::layout(p, batch);
  const hdd::Arenas A = arenas(p, L, ws);
  const hdd::SweepSub& sw = p.sweep;
  if (&per_depth == &p.down_all_lists && sw.height > 0 && sw.d_subs) {
    cudaError_t e =
        descent_levels(p, batch, A, sw.top_lists, sw.top_infos, sw.top_data, sw.d_top, u, u_stride, st, prof);
    if (e != cudaSuccess) return e;
    ProfScope ps(prof, hdd::kProfDescent, 0.0, st);
    const hdd::SubArgs g = sub_args(p, batch, A, true);
    return sw.fp64 ? hdd::launch_descent_sub<double>(g, sw.n_sub, sw.smem_desc, u, u_stride, st)
                   : hdd::launch_descent_sub<float>(g, sw.n_sub, sw.smem_desc, u, u_stride, st);
  }
  return descent_levels(p, batch, A, per_depth, p.lists, p.list_data, p.d_lists, u, u_stride, st, prof);
}

// Right-hand-side sweep (leaves to root) through the stored factors; plans with fused
// sweep subtrees run those first, then the heights above them.
cudaError_t run_forward(const hdd::Plan& p, int batch, void* ws, const hdd::Rhs& rhs, cudaStream_t st,
                        hdd::Profiler* prof) {
  const hdd::Layout L = hdd::layout(p, batch);
  const hdd::Arenas A = arenas(p, L, ws);
  const hdd::SweepSub& sw = p.sweep;
  int h0 = 0;
  if (sw.height > 0 && sw.d_subs) {
    ProfScope ps(prof, hdd::kProfForward, 0.0, st);
    const hdd::SubArgs g = sub_args(p, batch, A, false);
    cudaError_t e = sw.fp64 ? hdd::launch_forward_sub<double>(g, sw.n_sub, sw.smem_fwd, rhs, st)
                            : hdd::launch_forward_sub<float>(g, sw.n_sub, sw.smem_fwd, rhs, st);
    if (e != cudaSuccess) return e;
    h0 = sw.height + 1;
  }
  for (int h = h0; h <= p.height; ++h)
    for (int k = 0; k < 4; ++k) {
      const hdd::ListInfo& li = p.lists[p.fwd_lists[h][k]];
      if (li.n == 0) continue;
      if (k >= 2) {   // condensed leaves
        ProfScope ps(prof, hdd::kProfForward, 0.0, st);
        cudaError_t e = k == 2 ? hdd::launch_leaf_forward<double>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n,
                                                                  batch, A, rhs, st)
                               : hdd::launch_leaf_forward<float>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n,
                                                                 batch, A, rhs, st);
        if (e != cudaSuccess) return e;
        continue;
      }
      const bool cta = li.max_m >= kSweepCtaMinM;
      ProfScope ps(prof, hdd::kProfForward, 0.0, st);
      cudaError_t e;
      if (li.max_nf <= hdd::kTinyMax)
        e = k == 0 ? hdd::launch_forward_tiny<double>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs, st)
                   : hdd::launch_forward_tiny<float>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs, st);
      else if (mid_list(li))
        e = k == 0 ? hdd::launch_forward_mid<double>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs, st)
                   : hdd::launch_forward_mid<float>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs, st);
      else if (cta)
        e = k == 0 ? hdd::launch_forward<double>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs,
                                                 li.max_nf, st)
                   : hdd::launch_forward<float>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs,
                                                li.max_nf, st);
      else
        e = k == 0 ? hdd::launch_forward_warp<double>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs,
                                                      li.max_nf, li.max_m, st)
                   : hdd::launch_forward_warp<float>(p.d_nodes, p.d_maps, p.d_lists + li.off, li.n, batch, A, rhs,
                                                     li.max_nf, li.max_m, st);
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

hdd::FuncArgs func_args(const hdd::Plan& p, int batch, void* ws) {
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(ws);
  hdd::FuncArgs f{};
  f.nodes = p.d_nodes;
  f.maps = p.d_maps;
  f.batch = batch;
  f.N = p.N;
  f.A = arenas(p, L, ws);
  f.fmu = reinterpret_cast<double*>(w + L.fmu);
  f.n_nodes = (int64_t)p.nodes.size();
  f.lam = reinterpret_cast<double*>(w + L.lam);
  f.lam_stride = p.lam_stride;
  f.lam_off = p.d_lam_off;
  return f;
}

// Mean functionals (Sec. 5.1 Lemma; the algorithms of Sec. 5.2) of the observed
// nodes and their subtrees, leaves to root, through the stored factors; mu^f
// uses the stored y_g, i.e. the load of the last upsweep or right-hand-side sweep.
cudaError_t run_functional(const hdd::Plan& p, int batch, void* ws, cudaStream_t st, hdd::Profiler* prof) {
  hdd::FuncArgs f = func_args(p, batch, ws);
  for (int h = 0; h <= p.height; ++h)
    for (int k = 0; k < 4; ++k) {
      const hdd::ListInfo& li = p.lists[p.func_lists[h][k]];
      if (li.n == 0) continue;
      f.list = p.d_lists + li.off;
      f.nlist = li.n;
      ProfScope ps(prof, hdd::kProfFunc, 0.0, st);
      cudaError_t e;
      switch (k) {
        case 0: e = hdd::launch_func_warp<double>(f, li.max_nf, st); break;
        case 1: e = hdd::launch_func_warp<float>(f, li.max_nf, st); break;
        case 2: e = hdd::launch_func_leaf<double>(f, st); break;
        default: e = hdd::launch_func_leaf<float>(f, st); break;
      }
      if (e != cudaSuccess) return e;
    }
  return cudaSuccess;
}

// Subdomain means of every node of one vertex field per sample (Eq. mean; fathers
// from their sons as in Sec. 5.1).
cudaError_t run_means(const hdd::Plan& p, int batch, const double* u, int64_t u_stride, double* means,
                      cudaStream_t st) {
  const int64_t ms = (int64_t)p.nodes.size();
  cudaError_t e = cudaSuccess;
  for (int h = 0; h <= p.height && e == cudaSuccess; ++h) {
    const hdd::ListInfo& li = p.lists[p.height_lists[h]];
    e = h == 0 ? hdd::launch_leaf_means(p.d_nodes, p.d_lists + li.off, li.n, u, u_stride, p.N, means, ms, batch, st)
               : hdd::launch_father_means(p.d_nodes, p.d_lists + li.off, li.n, means, ms, batch, st);
  }
  return e;
}

// Mixed precision point solve: full descent, then ir_max_iter refinement steps
// (FP64 residual, sweep through the FP32/FP64 factors, update); the last step's
// descent is pruned to the observation paths and checked against ir_tol.
cudaError_t run_refined_solve(const hdd::Plan& p, int batch, void* ws, double* u_obs, cudaStream_t st,
                              hdd::Profiler* prof) {
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(ws);
  double* u = reinterpret_cast<double*>(w + L.u);
  double* r = reinterpret_cast<double*>(w + L.r);
  double* du = reinterpret_cast<double*>(w + L.du);
  const double* kappa = reinterpret_cast<const double*>(w + L.kappa);
  int32_t* status = reinterpret_cast<int32_t*>(w + L.status);
  double* dprev = reinterpret_cast<double*>(w + L.conv);   // zeroed by hdd_assemble
  const int64_t NN = (int64_t)p.N * p.N;
  const double load = p.h * p.h * p.f;
  const int K = p.ir_max_iter;
  cudaError_t e = cudaSuccess;
  // mean plans average the refined iterate over whole rectangles (Eq. mean), whose
  // Dirichlet vertices the descents never write: they hold g = 0
  if (p.obs_kind == HDD_OBS_MEANS && K > 0) e = cudaMemsetAsync(u, 0, (size_t)batch * NN * 8, st);
  if (e == cudaSuccess)
    e = run_descent(p, batch, ws, K > 0 ? p.down_all_lists : p.down_vis_lists, u, NN, st, prof);
  for (int it = 1; it <= K && e == cudaSuccess; ++it) {
    const bool last = it == K;
    {
      ProfScope ps(prof, hdd::kProfResidual, 0.0, st);
      e = hdd::launch_residual(kappa, p.n_t, u, NN, p.N, load, nullptr, 0, r, NN, batch, st);
    }
    if (e == cudaSuccess) e = run_forward(p, batch, ws, hdd::Rhs{r, NN, 0.0}, st, prof);
    if (e == cudaSuccess) e = run_descent(p, batch, ws, last ? p.down_vis_lists : p.down_all_lists, du, NN, st, prof);
    ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
    if (e == cudaSuccess && !last) e = hdd::launch_delta_obs(du, NN, p.d_obs, p.n_conv, dprev, batch, st);
    if (e == cudaSuccess && !last) e = hdd::launch_update(u, NN, du, NN, p.N, batch, st);
  }
  const bool means = p.obs_kind == HDD_OBS_MEANS;
  if (e == cudaSuccess) {
    ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
    // mean plans: the convergence test runs on the observed nodes' boundary unknowns
    double* out = means ? reinterpret_cast<double*>(w + L.conv_u) : u_obs;
    e = hdd::launch_final_obs(u, K > 0 ? du : nullptr, NN, p.d_obs, p.n_conv, K > 0 ? p.ir_tol : -1.0, dprev, out,
                              status, batch, st);
  }
  if (means && e == cudaSuccess) {
    // mean = Eq. mean of the refined iterate + the functional of the last correction
    // (its boundary values from the pruned descent, its load the last residual,
    // which the last right-hand-side sweep left in y_g); without refinement the
    // functional of the solution itself
    double* mfull = K > 0 ? reinterpret_cast<double*>(w + L.mfull) : nullptr;
    if (K > 0) {
      ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
      e = run_means(p, batch, u, NN, mfull, st);
    }
    if (e == cudaSuccess) e = run_functional(p, batch, ws, st, prof);
    if (e == cudaSuccess) {
      ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
      e = hdd::launch_mean_obs(func_args(p, batch, ws), p.d_obs_nodes, p.n_obs, K > 0 ? du : u, NN, mfull, u_obs,
                               st);
    }
  }
  return e;
}

// One load vector per sample through the stored factors (the operators of every
// node are computed once and applied to any right-hand side): right-hand-side
// sweep with b = c, full descent into u; mixed plans then take ir_max_iter FP64
// refinement steps over every unknown.
cudaError_t run_load_solve(const hdd::Plan& p, int batch, void* ws, const double* c, int64_t c_stride, double* u,
                           int64_t u_stride, cudaStream_t st, hdd::Profiler* prof) {
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(ws);
  double* r = reinterpret_cast<double*>(w + L.r);
  double* du = reinterpret_cast<double*>(w + L.du);
  const double* kappa = reinterpret_cast<const double*>(w + L.kappa);
  int32_t* status = reinterpret_cast<int32_t*>(w + L.status);
  double* dprev = reinterpret_cast<double*>(w + L.conv);
  const int64_t NN = (int64_t)p.N * p.N;
  cudaError_t e = run_forward(p, batch, ws, hdd::Rhs{c, c_stride, 0.0}, st, prof);
  if (e == cudaSuccess) e = run_descent(p, batch, ws, p.down_all_lists, u, u_stride, st, prof);
  if (p.precision != HDD_MIXED_FP32) return e;
  const int K = p.ir_max_iter;
  if (e == cudaSuccess && K > 0) e = cudaMemsetAsync(dprev, 0, (size_t)batch * 8, st);
  for (int it = 1; it <= K && e == cudaSuccess; ++it) {
    {
      ProfScope ps(prof, hdd::kProfResidual, 0.0, st);
      e = hdd::launch_residual(kappa, p.n_t, u, u_stride, p.N, 0.0, c, c_stride, r, NN, batch, st);
    }
    if (e == cudaSuccess) e = run_forward(p, batch, ws, hdd::Rhs{r, NN, 0.0}, st, prof);
    if (e == cudaSuccess) e = run_descent(p, batch, ws, p.down_all_lists, du, NN, st, prof);
    ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
    if (e == cudaSuccess) e = hdd::launch_update(u, u_stride, du, NN, p.N, batch, st);
    if (e == cudaSuccess) e = hdd::launch_conv_full(du, NN, u, u_stride, p.N, p.ir_tol, dprev, status, it == K, batch, st);
  }
  return e;
}

}  // namespace

extern "C" {

const char* hdd_status_string(hdd_status s) {
  switch (s) {
    case HDD_OK: return "ok";
    case HDD_EINVAL: return "invalid argument";
    case HDD_ENOMEM: return "out of memory";
    case HDD_ECUDA: return "CUDA error";
    case HDD_ENOTSPD: return "Schur block not positive definite";
    case HDD_ENOCONV: return "iterative refinement did not converge";
    case HDD_ETIMEOUT: return "device wait timed out";
    case HDD_ESTATE: return "operation needs a device plan";
  }
  return "unknown status";
}

const char* hdd_last_error(void) { return g_err.c_str(); }

hdd_status hdd_plan(const hdd_plan_desc* desc, hdd_plan_t* out) {
  if (!desc || !out) return fail_inval("NULL argument");
  *out = nullptr;
  hdd_plan_s* h = new (std::nothrow) hdd_plan_s;
  if (!h) return HDD_ENOMEM;
  std::string err;
  try {
    err = hdd::build_plan(*desc, h->p);
  } catch (const std::bad_alloc&) {
    delete h;
    g_err = "host allocation failed";
    return HDD_ENOMEM;
  } catch (...) {
    delete h;
    g_err = "plan construction failed";
    return HDD_EINVAL;
  }
  if (!err.empty()) {
    delete h;
    return fail_inval(err);
  }
  hdd::Plan& p = h->p;
  if (p.device >= 0) {
    if (!desc->kl_basis) {
      delete h;
      return fail_inval("kl_basis is NULL");
    }
    DeviceScope ds(p.device);
    if (ds.err != cudaSuccess) {
      delete h;
      return fail_cuda(ds.err, "cudaSetDevice");
    }
    cudaError_t e = configure_device(p.device);
    if (e == cudaSuccess) e = upload(&p.d_phi, desc->kl_basis, (size_t)p.n_t * p.n_z);
    if (e == cudaSuccess && p.precision == HDD_MIXED_FP32) {
      const size_t n = (size_t)p.n_t * p.n_z;
      std::vector<float> hi(n), lo(n);
      for (size_t i = 0; i < n; ++i) {
        hi[i] = (float)desc->kl_basis[i];
        lo[i] = (float)(desc->kl_basis[i] - (double)hi[i]);
      }
      e = upload(&p.d_phi_hi, hi.data(), n);
      if (e == cudaSuccess) e = upload(&p.d_phi_lo, lo.data(), n);
    }
    if (e == cudaSuccess) e = upload(&p.d_nodes, p.dev_nodes.data(), p.dev_nodes.size());
    if (e == cudaSuccess) e = upload(&p.d_maps, p.maps.data(), p.maps.size());
    if (e == cudaSuccess) e = upload(&p.d_lists, p.list_data.data(), p.list_data.size());
    if (e == cudaSuccess) e = upload(&p.d_obs, p.obs.data(), p.obs.size());
    if (e == cudaSuccess) e = upload(&p.d_fuse_soff, p.fuse_soff.data(), p.fuse_soff.size());
    if (e == cudaSuccess) e = upload(&p.d_lam_off, p.lam_off.data(), p.lam_off.size());
    if (e == cudaSuccess) e = upload(&p.d_obs_nodes, p.obs_nodes.data(), p.obs_nodes.size());
    if (e == cudaSuccess) e = upload_sweep(p.sweep);
    for (auto& fu : p.fusion)
      if (e == cudaSuccess && fu.height > 0) {
        e = upload(&fu.d_roots, fu.roots.data(), fu.roots.size());
        if (e == cudaSuccess) e = upload(&fu.d_nodes, fu.nodes.data(), fu.nodes.size());
      }
    if (e != cudaSuccess) {
      free_device(p);
      delete h;
      return e == cudaErrorMemoryAllocation ? (g_err = "device allocation failed", HDD_ENOMEM)
                                            : fail_cuda(e, "hdd_plan upload");
    }
  }
  *out = h;
  return HDD_OK;
}

hdd_status hdd_plan_destroy(hdd_plan_t plan) {
  if (!plan) return HDD_OK;
  if (plan->p.device >= 0) {
    DeviceScope ds(plan->p.device);
    free_device(plan->p);
    if (plan->prof) {
      hdd::Profiler* pr = static_cast<hdd::Profiler*>(plan->prof);
      for (cudaEvent_t e : pr->ev) cudaEventDestroy(e);
      delete pr;
      plan->prof = nullptr;
    }
  }
  delete plan;
  return HDD_OK;
}

hdd_status hdd_workspace_size(hdd_plan_t plan, int32_t batch, size_t* bytes) {
  if (!plan || !bytes) return fail_inval("NULL argument");
  if (batch < 1 || batch > 65535) return fail_inval("batch must be in 1..65535");
  *bytes = hdd::layout(plan->p, batch).total;
  return HDD_OK;
}

hdd_status hdd_assemble(hdd_plan_t plan, const double* Z, int32_t batch, void* workspace, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!Z) return fail_inval("Z is NULL");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(workspace);
  cudaError_t e = cudaMemsetAsync(w + L.status, 0, (size_t)batch * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w + L.conv, 0, (size_t)batch * 8, st);
  if (e == cudaSuccess) {
    ProfScope ps(profiler(plan), hdd::kProfKappa, 2.0 * p.n_t * p.n_z * batch, st);
    if (p.precision == HDD_MIXED_FP32)
      e = hdd::launch_kappa_df(p.d_phi_hi, p.d_phi_lo, Z, p.n_t, p.n_z, batch, reinterpret_cast<double*>(w + L.kappa),
                               reinterpret_cast<float*>(w + L.kappa32), p.n_t, st);
    else
      e = hdd::launch_kappa(p.d_phi, Z, p.n_t, p.n_z, batch, reinterpret_cast<double*>(w + L.kappa), nullptr, p.n_t,
                            st);
  }
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_assemble");
}

hdd_status hdd_upsweep(hdd_plan_t plan, int32_t batch, void* workspace, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  hdd::Rhs rhs{nullptr, 0, p.h * p.h * p.f};
  cudaError_t e = run_upsweep(p, batch, workspace, rhs, static_cast<cudaStream_t>(stream), profiler(plan));
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_upsweep");
}

hdd_status hdd_point_solve(hdd_plan_t plan, int32_t batch, void* workspace, double* u_obs, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!u_obs) return fail_inval("u_obs is NULL");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(workspace);
  double* u = reinterpret_cast<double*>(w + L.u);
  const int64_t NN = (int64_t)p.N * p.N;
  cudaError_t e;
  if (p.precision == HDD_MIXED_FP32) {
    e = run_refined_solve(p, batch, workspace, u_obs, st, profiler(plan));
  } else if (p.obs_kind == HDD_OBS_MEANS) {
    // descent to the observed nodes' ancestors only, then Eq. prop1 with the mean
    // functionals of the observed nodes (Sec. 5.1-5.2)
    e = run_descent(p, batch, workspace, p.down_vis_lists, u, NN, st, profiler(plan));
    if (e == cudaSuccess) e = run_functional(p, batch, workspace, st, profiler(plan));
    ProfScope ps(profiler(plan), hdd::kProfMisc, 0.0, st);
    if (e == cudaSuccess)
      e = hdd::launch_mean_obs(func_args(p, batch, workspace), p.d_obs_nodes, p.n_obs, u, NN, nullptr, u_obs, st);
  } else {
    e = run_descent(p, batch, workspace, p.down_vis_lists, u, NN, st, profiler(plan));
    ProfScope ps(profiler(plan), hdd::kProfMisc, 0.0, st);
    if (e == cudaSuccess) e = hdd::launch_gather_obs(u, NN, p.d_obs, p.n_obs, batch, u_obs, st);
  }
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_point_solve");
}

hdd_status hdd_loglik(hdd_plan_t plan, int32_t batch, void* workspace, const double* u_obs, const double* y,
                      int32_t y_per_sample, double* loglik, int32_t* sample_status, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!u_obs || !y || !loglik) return fail_inval("NULL argument");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(workspace);
  const int32_t* status = reinterpret_cast<const int32_t*>(w + L.status);
  cudaError_t e;
  {
    ProfScope ps(profiler(plan), hdd::kProfMisc, 0.0, st);
    e = hdd::launch_loglik(u_obs, p.n_obs, batch, y, y_per_sample ? 1 : 0, p.sigma, status, loglik, st);
  }
  if (e == cudaSuccess && sample_status)
    e = cudaMemcpyAsync(sample_status, status, (size_t)batch * 4, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_loglik");
}

hdd_status hdd_evaluate_host(hdd_plan_t plan, int32_t batch, void* workspace, const double* Z, const double* y,
                             int32_t y_per_sample, double* loglik, double* u_obs, int32_t* sample_status,
                             void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!Z || !y || !loglik) return fail_inval("NULL argument");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(workspace);
  double* dZ = reinterpret_cast<double*>(w + L.z);
  double* dy = reinterpret_cast<double*>(w + L.y);
  double* duobs = reinterpret_cast<double*>(w + L.uobs);
  double* dll = reinterpret_cast<double*>(w + L.ll);
  const size_t ny = (size_t)p.n_obs * (y_per_sample ? batch : 1);
  cudaError_t e = cudaMemcpyAsync(dZ, Z, (size_t)batch * p.n_z * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, ny * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_cuda(e, "hdd_evaluate_host copy in");
  if ((s = hdd_assemble(plan, dZ, batch, workspace, stream)) != HDD_OK) return s;
  if ((s = hdd_upsweep(plan, batch, workspace, stream)) != HDD_OK) return s;
  if ((s = hdd_point_solve(plan, batch, workspace, duobs, stream)) != HDD_OK) return s;
  if ((s = hdd_loglik(plan, batch, workspace, duobs, dy, y_per_sample, dll, nullptr, stream)) != HDD_OK) return s;
  e = cudaMemcpyAsync(loglik, dll, (size_t)batch * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && u_obs)
    e = cudaMemcpyAsync(u_obs, duobs, (size_t)batch * p.n_obs * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && sample_status)
    e = cudaMemcpyAsync(sample_status, w + L.status, (size_t)batch * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_evaluate_host");
}

hdd_status hdd_solve_loads(hdd_plan_t plan, int32_t batch, void* workspace, const double* c, int32_t n_loads,
                           double* u, int32_t* sample_status, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!c || !u) return fail_inval("c or u is NULL");
  if (n_loads < 1) return fail_inval("n_loads must be >= 1");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t NN = (int64_t)p.N * p.N;
  const int64_t stride = (int64_t)n_loads * NN;   // elements between samples of c and u
  cudaError_t e = cudaMemsetAsync(u, 0, (size_t)batch * stride * 8, st);   // Dirichlet vertices: g = 0
  for (int k = 0; k < n_loads && e == cudaSuccess; ++k)
    e = run_load_solve(p, batch, workspace, c + k * NN, stride, u + k * NN, stride, st, profiler(plan));
  if (e == cudaSuccess && sample_status)
    e = cudaMemcpyAsync(sample_status, static_cast<char*>(workspace) + hdd::layout(p, batch).status,
                        (size_t)batch * 4, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_solve_loads");
}

hdd_status hdd_data_scratch_size(hdd_plan_t plan, int32_t batch, size_t* bytes) {
  if (!plan || !bytes) return fail_inval("NULL argument");
  if (batch < 1 || batch > 65535) return fail_inval("batch must be in 1..65535");
  const size_t NN = (size_t)plan->p.N * plan->p.N;
  *bytes = (2 * (size_t)hdd::kData * batch * NN + 4 * (size_t)batch) * 8;
  return HDD_OK;
}

hdd_status hdd_solve_data(hdd_plan_t plan, int32_t batch, void* workspace, void* scratch, const double* c,
                          const double* f_coarse, const double* g, int32_t n_loads, double* u,
                          int32_t* sample_status, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  const hdd::Plan& p = plan->p;
  if (!u || !scratch) return fail_inval("u or scratch is NULL");
  if (reinterpret_cast<uintptr_t>(scratch) % 256 != 0) return fail_inval("scratch must be 256-byte aligned");
  if ((c == nullptr) == (f_coarse == nullptr)) return fail_inval("give exactly one of c and f_coarse");
  if (f_coarse && p.N % 2 == 0) return fail_inval("a coarse-grid load needs an odd N");
  if (n_loads < 1) return fail_inval("n_loads must be >= 1");
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  char* w = static_cast<char*>(workspace);
  const size_t NN = (size_t)p.N * p.N;
  hdd::DataArgs D{};
  D.nodes = p.d_nodes;
  D.maps = p.d_maps;
  D.A = arenas(p, L, workspace);
  D.N = p.N;
  D.batch = batch;
  D.n_loads = n_loads;
  D.h2 = p.h * p.h;
  D.u = u;
  D.d = static_cast<double*>(scratch);
  D.r = D.d + (size_t)hdd::kData * batch * NN;
  D.conv = D.r + (size_t)hdd::kData * batch * NN;
  D.status = reinterpret_cast<int32_t*>(w + L.status);
  const double* kappa = reinterpret_cast<const double*>(w + L.kappa);
  const int K = p.precision == HDD_MIXED_FP32 ? p.ir_max_iter : 0;
  hdd::Profiler* prof = profiler(plan);
  cudaError_t e = cudaMemsetAsync(D.conv, 0, (size_t)batch * 4 * 8, st);
  for (int k0 = 0; k0 < n_loads && e == cudaSuccess; k0 += hdd::kData) {
    D.nk = std::min(hdd::kData, n_loads - k0);
    e = hdd::launch_data_init(D, g, k0, st);
    for (int it = 0; it <= K && e == cudaSuccess; ++it) {
      {
        ProfScope ps(prof, hdd::kProfResidual, 0.0, st);
        e = hdd::launch_data_residual(D, kappa, p.n_t, c, f_coarse, k0, st);
      }
      for (int h = 0; h <= p.height && e == cudaSuccess; ++h)   // leaves to root, every node
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
          const hdd::ListInfo& li = p.lists[p.fwd_lists[h][k]];
          if (li.n == 0) continue;
          ProfScope ps(prof, hdd::kProfForward, 0.0, st);
          const int32_t* l = p.d_lists + li.off;
          e = k == 0 ? hdd::launch_data_sweep<double>(D, l, li.n, li.max_nf, li.max_m, false, st)
            : k == 1 ? hdd::launch_data_sweep<float>(D, l, li.n, li.max_nf, li.max_m, false, st)
            : k == 2 ? hdd::launch_data_leaf<double>(D, l, li.n, false, st)
                     : hdd::launch_data_leaf<float>(D, l, li.n, false, st);
        }
      for (int d = 0; d <= p.depth && e == cudaSuccess; ++d)    // root to leaves, every node
        for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
          const hdd::ListInfo& li = p.lists[p.down_all_lists[d][k]];
          if (li.n == 0) continue;
          ProfScope ps(prof, hdd::kProfDescent, 0.0, st);
          const int32_t* l = p.d_lists + li.off;
          if (k == 0)
            e = p.nodes[p.list_data[li.off]].fp64 ? hdd::launch_data_sweep<double>(D, l, li.n, li.max_nf, li.max_m, true, st)
                                                  : hdd::launch_data_sweep<float>(D, l, li.n, li.max_nf, li.max_m, true, st);
          else
            e = k == 1 ? hdd::launch_data_leaf<double>(D, l, li.n, true, st)
                       : hdd::launch_data_leaf<float>(D, l, li.n, true, st);
        }
      if (e == cudaSuccess) {
        ProfScope ps(prof, hdd::kProfMisc, 0.0, st);
        e = hdd::launch_data_update(D, k0, p.ir_tol, it == K, it > 0, st);
      }
    }
  }
  if (e == cudaSuccess && sample_status)
    e = cudaMemcpyAsync(sample_status, D.status, (size_t)batch * 4, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_solve_data");
}

hdd_status hdd_subdomain_means(hdd_plan_t plan, int32_t batch, const double* u, int64_t u_stride, double* means,
                               void* stream) {
  if (!plan) return fail_inval("plan is NULL");
  const hdd::Plan& p = plan->p;
  if (p.device < 0) {
    g_err = "host-only plan";
    return HDD_ESTATE;
  }
  if (batch < 1 || batch > 65535) return fail_inval("batch must be in 1..65535");
  if (!u || !means) return fail_inval("u or means is NULL");
  if (u_stride < (int64_t)p.N * p.N) return fail_inval("u_stride must be >= N*N");
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ProfScope ps(profiler(plan), hdd::kProfMisc, 0.0, st);
  const cudaError_t e = run_means(p, batch, u, u_stride, means, st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_subdomain_means");
}

hdd_status hdd_mean_functionals(hdd_plan_t plan, int32_t batch, void* workspace, double* lambda_g, double* mu_f,
                                void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  const hdd::Plan& p = plan->p;
  if (p.obs_kind != HDD_OBS_MEANS) {
    g_err = "the plan does not observe subdomain means";
    return HDD_ESTATE;
  }
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const hdd::Layout L = hdd::layout(p, batch);
  const char* w = static_cast<const char*>(workspace);
  cudaError_t e = cudaSuccess;
  if (lambda_g && p.lam_stride > 0)
    e = cudaMemcpyAsync(lambda_g, w + L.lam, (size_t)batch * p.lam_stride * 8, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && mu_f)
    e = cudaMemcpyAsync(mu_f, w + L.fmu, (size_t)batch * p.nodes.size() * 8, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_mean_functionals");
}

hdd_status hdd_kappa(hdd_plan_t plan, int32_t batch, void* workspace, double* kappa, void* stream) {
  hdd_status s = check_call(plan, batch, workspace);
  if (s != HDD_OK) return s;
  if (!kappa) return fail_inval("kappa is NULL");
  const hdd::Plan& p = plan->p;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  const hdd::Layout L = hdd::layout(p, batch);
  cudaError_t e = cudaMemcpyAsync(kappa, static_cast<char*>(workspace) + L.kappa, (size_t)batch * p.n_t * 8,
                                  cudaMemcpyDeviceToDevice, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HDD_OK : fail_cuda(e, "hdd_kappa");
}

hdd_status hdd_set_sweep_fusion(hdd_plan_t plan, int32_t max_height) {
  if (!plan) return fail_inval("plan is NULL");
  if (max_height < 0 || max_height > hdd::kSweepMaxHeight) return fail_inval("max_height must be in 0..6");
  hdd::Plan& p = plan->p;
  hdd::SweepSub old = std::move(p.sweep);
  p.sweep_max_height = max_height;
  hdd::build_sweep(p, max_height);
  if (p.device < 0) return HDD_OK;
  DeviceScope ds(p.device);
  if (ds.err != cudaSuccess) return fail_cuda(ds.err, "cudaSetDevice");
  free_sweep(old);
  const cudaError_t e = upload_sweep(p.sweep);
  if (e != cudaSuccess) {
    free_sweep(p.sweep);
    p.sweep = hdd::SweepSub{};   // the level-by-level sweeps stay usable
    return e == cudaErrorMemoryAllocation ? (g_err = "device allocation failed", HDD_ENOMEM)
                                          : fail_cuda(e, "hdd_set_sweep_fusion upload");
  }
  return HDD_OK;
}

hdd_status hdd_set_wait_bound(hdd_plan_t plan, uint32_t polls, int32_t stall_node, int32_t stall_sample) {
  if (!plan) return fail_inval("plan is NULL");
  if (polls == 0) return fail_inval("polls must be >= 1");
  hdd::Plan& p = plan->p;
  if (stall_node < -1 || stall_node >= (int32_t)p.nodes.size()) return fail_inval("stall_node out of range");
  if (stall_sample < -1) return fail_inval("stall_sample out of range");
  p.wait_limit = polls;
  p.stall_node = stall_node;
  p.stall_sample = stall_node < 0 ? -1 : stall_sample;
  return HDD_OK;
}

hdd_status hdd_profile_begin(hdd_plan_t plan) {
  if (!plan) return fail_inval("plan is NULL");
  if (plan->p.device < 0) {
    g_err = "host-only plan";
    return HDD_ESTATE;
  }
  if (!plan->prof) plan->prof = new (std::nothrow) hdd::Profiler;
  if (!plan->prof) return HDD_ENOMEM;
  hdd::Profiler* pr = static_cast<hdd::Profiler*>(plan->prof);
  pr->used = 0;
  pr->on = true;
  return HDD_OK;
}

hdd_status hdd_profile_end(hdd_plan_t plan, hdd_kernel_stat_t* stats, int32_t max_stats, int32_t* n_stats) {
  if (!plan || !plan->prof) return fail_inval("profiling was not started");
  hdd::Profiler* pr = static_cast<hdd::Profiler*>(plan->prof);
  pr->on = false;
  static const char* names[hdd::kProfCount] = {"kappa", "front_warp", "front_small", "front_fill", "potrf", "trsm",
                                                "syrk_simt", "syrk_tc", "syrk_rhs", "forward", "descent",
                                                "residual", "misc", "subtree", "leaf_front", "chol_trsm",
                                                "functional"};
  int launches[hdd::kProfCount] = {};
  double ms[hdd::kProfCount] = {}, fl[hdd::kProfCount] = {};
  DeviceScope ds(plan->p.device);
  for (size_t k = 0; k < pr->used; ++k) {
    float t = 0.0f;
    cudaError_t e = cudaEventSynchronize(pr->ev[2 * k + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pr->ev[2 * k], pr->ev[2 * k + 1]);
    if (e != cudaSuccess) return fail_cuda(e, "hdd_profile_end");
    launches[pr->fam[k]] += 1;
    ms[pr->fam[k]] += t;
    fl[pr->fam[k]] += pr->flops[k];
  }
  pr->used = 0;
  int n = 0;
  for (int f = 0; f < hdd::kProfCount; ++f) {
    if (!launches[f]) continue;
    if (stats && n < max_stats) {
      std::strncpy(stats[n].name, names[f], sizeof(stats[n].name) - 1);
      stats[n].name[sizeof(stats[n].name) - 1] = 0;
      stats[n].launches = launches[f];
      stats[n].ms = ms[f];
      stats[n].flops = fl[f];
    }
    ++n;
  }
  if (n_stats) *n_stats = n;
  return HDD_OK;
}

hdd_status hdd_plan_info(hdd_plan_t plan, hdd_plan_info_t* info) {
  if (!plan || !info) return fail_inval("NULL argument");
  const hdd::Plan& p = plan->p;
  info->n_nodes = (int32_t)p.nodes.size();
  info->n_leaves = p.n_leaves;
  info->depth = p.depth;
  info->height = p.height;
  info->n_visited = p.n_visited;
  info->max_front = p.max_front;
  info->flops_upsweep = p.flops_up;
  info->flops_point_solve = p.flops_down;
  info->factor_bytes = (double)p.f64_stride * 8 + (double)p.f32_stride * 4;
  info->schur_bytes = (double)p.s64_stride * 8 + (double)p.s32_stride * 4;
  info->bytes_upsweep_tiny = p.by_tiny;
  info->bytes_upsweep_small = p.by_small;
  info->bytes_upsweep_large = p.by_large;
  info->bytes_upsweep_fused = p.by_fused;
  info->bytes_forward = p.by_fwd;
  info->bytes_descent_all = p.by_desc_all;
  info->bytes_descent_visited = p.by_desc_vis;
  info->bytes_residual = p.by_residual;
  info->bytes_assemble = p.by_assemble;
  info->bytes_kl_basis = p.by_kl_basis;
  info->bytes_upsweep_leaf = p.by_leaf;
  info->n_condensed_leaves = 0;
  for (const hdd::Node& nd : p.nodes) info->n_condensed_leaves += nd.linv;
  int up = 0, down = 0;
  for (int h = 0; h <= p.height; ++h)
    for (int kind = 0; kind < 8; ++kind) up += hdd::step_launches(kind, p.lists[p.step_lists[h][kind]]);
  for (const auto& fu : p.fusion) up += fu.height > 0;
  int down_all = 0, fwd = 0;
  for (int d = 0; d <= p.depth; ++d)
    for (int kind = 0; kind < 3; ++kind) {
      down += p.lists[p.down_vis_lists[d][kind]].n > 0;
      down_all += p.lists[p.down_all_lists[d][kind]].n > 0;
    }
  const hdd::SweepSub& sw = p.sweep;
  for (int h = sw.height > 0 ? sw.height + 1 : 0; h <= p.height; ++h)
    for (int k = 0; k < 4; ++k) fwd += p.lists[p.fwd_lists[h][k]].n > 0;
  if (sw.height > 0) {   // fused sweep subtrees: one launch each way, plus the levels above
    fwd += 1;
    down_all = 1;
    for (const auto& l : sw.top_lists)
      for (int kind = 0; kind < 3; ++kind) down_all += sw.top_infos[l[kind]].n > 0;
  }
  info->sweep_fuse_height = sw.height;
  int solve = down + 1;
  int func = 0;
  for (int h = 0; h <= p.height && p.obs_kind == HDD_OBS_MEANS; ++h)
    for (int k = 0; k < 4; ++k) func += p.lists[p.func_lists[h][k]].n > 0;
  if (p.precision == HDD_MIXED_FP32) {
    const int K = p.ir_max_iter;
    solve = (K > 0 ? down_all : down) + 1;
    for (int it = 1; it <= K; ++it) solve += 1 + fwd + (it == K ? down : down_all) + (it == K ? 0 : 2);
    if (p.obs_kind == HDD_OBS_MEANS) solve += func + 1 + (K > 0 ? p.height + 1 : 0);
  } else if (p.obs_kind == HDD_OBS_MEANS) {
    solve += func;
  }
  info->launches_upsweep = up;
  info->launches_evaluate = 1 + up + solve + 1;
  return HDD_OK;
}

hdd_status hdd_node_info(hdd_plan_t plan, int32_t node, hdd_node_info_t* info) {
  if (!plan || !info) return fail_inval("NULL argument");
  const hdd::Plan& p = plan->p;
  if (node < 0 || node >= (int32_t)p.nodes.size()) return fail_inval("node out of range");
  const hdd::Node& nd = p.nodes[node];
  info->x0 = nd.x0; info->x1 = nd.x1; info->y0 = nd.y0; info->y1 = nd.y1;
  info->parent = nd.parent; info->child0 = nd.child[0]; info->child1 = nd.child[1];
  info->depth = nd.depth; info->height = nd.height;
  info->m = nd.m; info->b = nd.b;
  info->visited = nd.visited ? 1 : 0;
  return HDD_OK;
}

hdd_status hdd_node_indices(hdd_plan_t plan, int32_t node, int32_t* gamma, int32_t* bnd) {
  if (!plan) return fail_inval("NULL argument");
  const hdd::Plan& p = plan->p;
  if (node < 0 || node >= (int32_t)p.nodes.size()) return fail_inval("node out of range");
  const hdd::Node& nd = p.nodes[node];
  if (gamma) std::memcpy(gamma, nd.gamma.data(), nd.gamma.size() * 4);
  if (bnd) std::memcpy(bnd, nd.bnd.data(), nd.bnd.size() * 4);
  return HDD_OK;
}

}  // extern "C"
