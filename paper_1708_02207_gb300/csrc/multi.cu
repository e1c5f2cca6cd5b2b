// Uneven batches: several plans (grids, KL bases, observation sets, precisions)
// whose "Leaves to Root" (Sec. 3.4) runs as one launch per tree height and front
// class over the nodes of every plan.
//
// The plans' node descriptors and index maps are concatenated into one table
// (children and map offsets shifted), and every list of one height and class
// holds the nodes of all plans at that height above their leaves.  A CTA reads
// its node, looks up the node's plan, and takes that plan's workspace arenas,
// coefficient field, load, status words, grid size and batch from a small table
// of parts (bind_plan): the per-sample arithmetic is exactly that of the plan run
// alone, so each sample's result does not depend on the batch it ran in.  A
// plan's list joins the merged list of the same launch choices: the large fronts'
// path (fused POTRF + TRSM or the blocked kernels, by the largest interface), the
// grouped kernel's warps per front (by the largest front), and the batch class
// (the batch's power of two): a merged launch is configured as each of its plans'
// own launch would be, and its grid, sized by the largest batch of its plans,
// wastes at most half its CTAs on samples beyond a plan's batch (they return at
// once).  Assembly, the point solve and the likelihood stay per plan (a handful of
// launches each).
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <new>
#include <string>
#include <vector>

#include "launch.h"
#include "plan.h"

namespace hdd {
hdd_status set_error(hdd_status status, const std::string& msg);
}

struct hdd_multi_s {
  int device = -1;
  std::vector<hdd_plan_t> plans;   // not owned
  std::vector<int> batches;
  std::vector<void*> ws;
  int height = 0, max_batch = 0;
  // launch order: per height, front class and path class; flops summed over the plans' samples
  std::vector<hdd::ListInfo> lists;
  std::vector<int> kinds;
  std::vector<int> list_batch;   // the largest batch of the plans in each list (its grid)
  std::vector<int32_t> list_data;
  hdd::NodeDev* d_nodes = nullptr;
  int32_t* d_maps = nullptr;
  int32_t* d_plan_of = nullptr;
  int32_t* d_lists = nullptr;
  hdd::PlanDev* d_parts = nullptr;
  int launches_upsweep = 0;
  // per plan a stream for the per-plan phases (forked from and joined to the
  // caller's stream by events), so that the plans' small launches overlap
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
};

namespace {

void free_multi(hdd_multi_s& m) {
  for (cudaStream_t st : m.streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : m.done) cudaEventDestroy(ev);
  if (m.fork) cudaEventDestroy(m.fork);
  m.streams.clear();
  m.done.clear();
  m.fork = nullptr;
  cudaFree(m.d_nodes);
  cudaFree(m.d_maps);
  cudaFree(m.d_plan_of);
  cudaFree(m.d_lists);
  cudaFree(m.d_parts);
  m.d_nodes = nullptr; m.d_maps = nullptr; m.d_plan_of = nullptr; m.d_lists = nullptr; m.d_parts = nullptr;
}

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  cudaError_t e = cudaMalloc((void**)dst, (n ? n : 1) * sizeof(T));
  if (e == cudaSuccess && n) e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

struct DevScope {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DevScope(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
  }
  ~DevScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

hdd_status cuda_fail(cudaError_t e, const char* where) {
  return hdd::set_error(HDD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

hdd_status hdd_multi_create(const hdd_plan_t* plans, int32_t n_plans, const int32_t* batches,
                            void* const* workspaces, hdd_multi_t* out) {
  if (!out) return hdd::set_error(HDD_EINVAL, "out is NULL");
  *out = nullptr;
  if (!plans || !batches || !workspaces || n_plans < 1)
    return hdd::set_error(HDD_EINVAL, "plans, batches and workspaces must hold n_plans >= 1 entries");
  hdd_multi_s* m = new (std::nothrow) hdd_multi_s;
  if (!m) return HDD_ENOMEM;
  for (int q = 0; q < n_plans; ++q) {
    const hdd_plan_t pl = plans[q];
    std::string bad;
    if (!pl) bad = "a plan is NULL";
    else if (pl->p.device < 0) bad = "a plan is host-only";
    else if (q > 0 && pl->p.device != plans[0]->p.device) bad = "plans on different devices";
    else if (pl->p.fusion[0].height || pl->p.fusion[1].height) bad = "plans with fused subtrees are not supported";
    else if (batches[q] < 1 || batches[q] > 65535) bad = "batch must be in 1..65535";
    else if (!workspaces[q] || reinterpret_cast<uintptr_t>(workspaces[q]) % 256 != 0)
      bad = "workspaces must be non-NULL and 256-byte aligned";
    if (!bad.empty()) {
      delete m;
      return hdd::set_error(HDD_EINVAL, bad);
    }
    m->plans.push_back(pl);
    m->batches.push_back(batches[q]);
    m->ws.push_back(workspaces[q]);
    m->height = std::max(m->height, pl->p.height);
    m->max_batch = std::max(m->max_batch, (int)batches[q]);
  }
  m->device = plans[0]->p.device;

  // concatenated node table and maps (children and map offsets shifted), node -> plan
  std::vector<hdd::NodeDev> nodes;
  std::vector<int32_t> maps, plan_of;
  std::vector<int64_t> node_base;
  for (int q = 0; q < n_plans; ++q) {
    const hdd::Plan& p = plans[q]->p;
    const int64_t nb = (int64_t)nodes.size(), mb = (int64_t)maps.size();
    if (mb + (int64_t)p.maps.size() > (int64_t)INT32_MAX || nb + (int64_t)p.dev_nodes.size() > (int64_t)INT32_MAX) {
      delete m;
      return hdd::set_error(HDD_EINVAL, "the plans' tables are too large for one launch");
    }
    node_base.push_back(nb);
    for (hdd::NodeDev d : p.dev_nodes) {
      if (d.child0 >= 0) d.child0 += (int32_t)nb;
      if (d.child1 >= 0) d.child1 += (int32_t)nb;
      d.map_off += (int32_t)mb;
      d.up_off += (int32_t)mb;
      nodes.push_back(d);
      plan_of.push_back(q);
    }
    maps.insert(maps.end(), p.maps.begin(), p.maps.end());
  }
  // per height above the leaves, front class and path class: the nodes of every plan
  // (path class of a large-front list: fused POTRF + TRSM for interfaces of at most 32
  // columns, or 64 in FP32 with two diagonal blocks, else the blocked kernels)
  auto launch_class = [&](int kind, const hdd::ListInfo& li, int batch) {
    int path = 0;
    if (kind == 2) path = li.max_m <= 32 ? 0 : 2;
    if (kind == 5) path = li.max_m <= 32 ? 0 : (li.max_m <= 64 ? 1 : 2);
    const bool grouped = kind == 0 || kind == 1 || kind == 3 || kind == 4;
    const int warps = grouped ? hdd::group_warps(li.max_nf, kind < 3) : 0;
    int bcls = 0;
    while ((2 << bcls) <= batch) ++bcls;   // floor(log2(batch))
    return (path * 16 + warps) * 32 + bcls;
  };
  for (int h = 0; h <= m->height; ++h)
    for (int kind = 0; kind < 8; ++kind) {
      std::vector<int> classes;
      for (int q = 0; q < n_plans; ++q) {
        const hdd::Plan& p = plans[q]->p;
        if (h > p.height) continue;
        const hdd::ListInfo& li = p.lists[p.step_lists[h][kind]];
        if (li.n == 0) continue;
        const int c = launch_class(kind, li, batches[q]);
        if (std::find(classes.begin(), classes.end(), c) == classes.end()) classes.push_back(c);
      }
      for (int cls : classes) {
        hdd::ListInfo L;
        L.off = (int64_t)m->list_data.size();
        int lbatch = 0;
        for (int q = 0; q < n_plans; ++q) {
          const hdd::Plan& p = plans[q]->p;
          if (h > p.height) continue;
          const hdd::ListInfo& li = p.lists[p.step_lists[h][kind]];
          if (li.n == 0 || launch_class(kind, li, batches[q]) != cls) continue;
          lbatch = std::max(lbatch, (int)batches[q]);
          for (int k = 0; k < li.n; ++k) m->list_data.push_back((int32_t)(node_base[q] + p.list_data[li.off + k]));
          L.n += li.n;
          L.max_nf = std::max(L.max_nf, li.max_nf);
          L.max_m = std::max(L.max_m, li.max_m);
          L.max_b = std::max(L.max_b, li.max_b);
          L.max_rect = std::max(L.max_rect, li.max_rect);
          L.fl_chol += li.fl_chol * batches[q];
          L.fl_trsm += li.fl_trsm * batches[q];
          L.fl_syrk += li.fl_syrk * batches[q];
          L.fl_rhs += li.fl_rhs * batches[q];
        }
        if (L.n == 0) continue;
        m->lists.push_back(L);
        m->kinds.push_back(kind);
        m->list_batch.push_back(lbatch);
        m->launches_upsweep += hdd::step_launches(kind, L);
      }
    }
  std::vector<hdd::PlanDev> parts;
  for (int q = 0; q < n_plans; ++q) parts.push_back(hdd::plan_part(plans[q]->p, batches[q], workspaces[q]));

  DevScope ds(m->device);
  cudaError_t e = ds.err;
  if (e == cudaSuccess) e = upload(&m->d_nodes, nodes.data(), nodes.size());
  if (e == cudaSuccess) e = upload(&m->d_maps, maps.data(), maps.size());
  if (e == cudaSuccess) e = upload(&m->d_plan_of, plan_of.data(), plan_of.size());
  if (e == cudaSuccess) e = upload(&m->d_lists, m->list_data.data(), m->list_data.size());
  if (e == cudaSuccess) e = upload(&m->d_parts, parts.data(), parts.size());
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming);
  for (int q = 0; q < n_plans && e == cudaSuccess; ++q) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) m->streams.push_back(st);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) m->done.push_back(ev);
  }
  if (e != cudaSuccess) {
    free_multi(*m);
    delete m;
    return e == cudaErrorMemoryAllocation ? hdd::set_error(HDD_ENOMEM, "device allocation failed")
                                          : cuda_fail(e, "hdd_multi_create");
  }
  *out = m;
  return HDD_OK;
}

hdd_status hdd_multi_destroy(hdd_multi_t multi) {
  if (!multi) return HDD_OK;
  {
    DevScope ds(multi->device);
    free_multi(*multi);
  }
  delete multi;
  return HDD_OK;
}

hdd_status hdd_multi_upsweep(hdd_multi_t multi, void* stream) {
  if (!multi) return hdd::set_error(HDD_EINVAL, "multi is NULL");
  DevScope ds(multi->device);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // defaults from the first plan; every kernel rebinds them from its node's plan
  hdd::StepArgs a{};
  const hdd::PlanDev p0 = hdd::plan_part(multi->plans[0]->p, multi->batches[0], multi->ws[0]);
  a.nodes = multi->d_nodes;
  a.maps = multi->d_maps;
  a.batch = multi->max_batch;
  a.N = p0.N;
  a.kappa = p0.kappa;
  a.kappa32 = p0.kappa32;
  a.kap_stride = p0.kap_stride;
  a.rhs = p0.rhs;
  a.arenas = p0.arenas;
  a.status = p0.status;
  a.prof = nullptr;
  a.wait_limit = 1u << 24;
  a.stall_node = a.stall_sample = -1;
  a.plans = multi->d_parts;
  a.plan_of = multi->d_plan_of;
  for (size_t k = 0; k < multi->lists.size(); ++k) {
    const hdd::ListInfo& li = multi->lists[k];
    a.list = multi->d_lists + li.off;
    a.batch = multi->list_batch[k];
    hdd::set_list(a, li, 1.0);
    const cudaError_t e = hdd::launch_step(multi->kinds[k], a, st);
    if (e != cudaSuccess) return cuda_fail(e, "hdd_multi_upsweep");
  }
  return HDD_OK;
}

hdd_status hdd_multi_evaluate(hdd_multi_t multi, const double* const* Z, const double* const* y,
                              const int32_t* y_per_sample, double* const* loglik, double* const* u_obs,
                              int32_t* const* sample_status, void* stream) {
  if (!multi) return hdd::set_error(HDD_EINVAL, "multi is NULL");
  if (!Z || !y || !y_per_sample || !loglik || !u_obs)
    return hdd::set_error(HDD_EINVAL, "Z, y, y_per_sample, loglik and u_obs must be arrays of n_plans pointers");
  const int n = (int)multi->plans.size();
  DevScope ds(multi->device);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // fork: every plan stream starts after the caller's earlier work; join: the
  // caller's stream continues after every plan stream
  auto fork = [&]() {
    cudaError_t e = cudaEventRecord(multi->fork, st);
    for (int q = 0; q < n && e == cudaSuccess; ++q) e = cudaStreamWaitEvent(multi->streams[q], multi->fork, 0);
    return e;
  };
  auto join = [&]() {
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
      e = cudaEventRecord(multi->done[q], multi->streams[q]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, multi->done[q], 0);
    }
    return e;
  };
  hdd_status s;
  cudaError_t e = fork();
  if (e != cudaSuccess) return cuda_fail(e, "hdd_multi_evaluate fork");
  for (int q = 0; q < n; ++q)
    if ((s = hdd_assemble(multi->plans[q], Z[q], multi->batches[q], multi->ws[q], multi->streams[q])) != HDD_OK)
      return s;
  if ((e = join()) != cudaSuccess) return cuda_fail(e, "hdd_multi_evaluate join");
  if ((s = hdd_multi_upsweep(multi, stream)) != HDD_OK) return s;
  if ((e = fork()) != cudaSuccess) return cuda_fail(e, "hdd_multi_evaluate fork");
  for (int q = 0; q < n; ++q) {
    cudaStream_t sq = multi->streams[q];
    if ((s = hdd_point_solve(multi->plans[q], multi->batches[q], multi->ws[q], u_obs[q], sq)) != HDD_OK) return s;
    if ((s = hdd_loglik(multi->plans[q], multi->batches[q], multi->ws[q], u_obs[q], y[q], y_per_sample[q],
                        loglik[q], sample_status ? sample_status[q] : nullptr, sq)) != HDD_OK)
      return s;
  }
  if ((e = join()) != cudaSuccess) return cuda_fail(e, "hdd_multi_evaluate join");
  return HDD_OK;
}

// A captured evaluation: the instantiated CUDA graph of one hdd_multi_evaluate.
struct hdd_graph_s {
  int device = -1;
  cudaGraphExec_t exec = nullptr;
};

hdd_status hdd_multi_capture(hdd_multi_t multi, const double* const* Z, const double* const* y,
                             const int32_t* y_per_sample, double* const* loglik, double* const* u_obs,
                             int32_t* const* sample_status, hdd_graph_t* out) {
  if (!multi || !out) return hdd::set_error(HDD_EINVAL, "multi and out must not be NULL");
  *out = nullptr;
  DevScope ds(multi->device);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "cudaSetDevice");
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "hdd_multi_capture stream");
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "hdd_multi_capture begin");
  }
  // the plan streams join the capture through the fork event and leave it through the
  // join events, exactly as they order a direct call after the caller's stream
  const hdd_status s = hdd_multi_evaluate(multi, Z, y, y_per_sample, loglik, u_obs, sample_status, cs);
  cudaGraph_t graph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(cs, &graph);   // ended whatever happened inside
  cudaGraphExec_t exec = nullptr;
  if (s == HDD_OK && ee == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (s != HDD_OK) return s;
  if (ee != cudaSuccess) return cuda_fail(ee, "hdd_multi_capture end");
  if (e != cudaSuccess) return cuda_fail(e, "hdd_multi_capture instantiate");
  hdd_graph_s* g = new (std::nothrow) hdd_graph_s;
  if (!g) {
    cudaGraphExecDestroy(exec);
    return hdd::set_error(HDD_ENOMEM, "host allocation failed");
  }
  g->device = multi->device;
  g->exec = exec;
  *out = g;
  return HDD_OK;
}

hdd_status hdd_graph_launch(hdd_graph_t graph, void* stream) {
  if (!graph) return hdd::set_error(HDD_EINVAL, "graph is NULL");
  DevScope ds(graph->device);
  if (ds.err != cudaSuccess) return cuda_fail(ds.err, "cudaSetDevice");
  const cudaError_t e = cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? HDD_OK : cuda_fail(e, "hdd_graph_launch");
}

hdd_status hdd_graph_destroy(hdd_graph_t graph) {
  if (!graph) return HDD_OK;
  {
    DevScope ds(graph->device);
    cudaGraphExecDestroy(graph->exec);
  }
  delete graph;
  return HDD_OK;
}

hdd_status hdd_multi_info(hdd_multi_t multi, int32_t* launches_upsweep, int32_t* launches_evaluate) {
  if (!multi) return hdd::set_error(HDD_EINVAL, "multi is NULL");
  if (launches_upsweep) *launches_upsweep = multi->launches_upsweep;
  if (launches_evaluate) {
    int total = multi->launches_upsweep;
    for (hdd_plan_t pl : multi->plans) {
      hdd_plan_info_t info;
      hdd_plan_info(pl, &info);
      total += info.launches_evaluate - info.launches_upsweep;   // assembly, point solve, likelihood
    }
    *launches_evaluate = total;
  }
  return HDD_OK;
}

}  // extern "C"
