// Host-side launchers of the HDD kernels (one translation unit per kernel family).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace hdd {

// Optional per-kernel timing (host side): CUDA event pairs recorded on the
// launching stream around each kernel, tagged with a kernel family and the
// algorithmic flops of the launch.  Owned by a plan; not thread-safe.
enum ProfFamily {
  kProfKappa, kProfFrontWarp, kProfFrontSmall, kProfFill, kProfPotrf, kProfTrsm, kProfSyrk, kProfSyrkTc,
  kProfSyrkRhs, kProfForward, kProfDescent, kProfResidual, kProfMisc, kProfFused, kProfLeaf, kProfCholTrsm,
  kProfFunc, kProfCount
};
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;       // 2 per record
  std::vector<int> fam;
  std::vector<double> flops;
  size_t used = 0;
  void begin(int family, double fl, cudaStream_t st) {
    if (!on) return;
    if (2 * used + 2 > ev.size()) {
      for (int k = 0; k < 64; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        ev.push_back(e);
      }
    }
    if (fam.size() <= used) { fam.resize(used + 1); flops.resize(used + 1); }
    fam[used] = family;
    flops[used] = fl;
    cudaEventRecord(ev[2 * used], st);
  }
  void end(cudaStream_t st) {
    if (!on || 2 * used + 2 > ev.size()) return;
    cudaEventRecord(ev[2 * used + 1], st);
    ++used;
  }
};

// One plan's part of a launch over several plans (hdd_multi_*): the workspace
// arenas, coefficient field, status words, load and sizes of that plan's batch.
struct PlanDev {
  Arenas arenas;
  const double* kappa;
  const float* kappa32;
  int64_t kap_stride;
  int32_t* status;
  Rhs rhs;
  int N, batch;
};

struct StepArgs {
  const NodeDev* nodes;
  const int32_t* maps;
  const int32_t* list;     // device node indices
  int nlist;
  int batch;
  int N;
  const double* kappa;     // [batch x n_t]
  const float* kappa32;    // FP32 copy (mixed plans) or nullptr
  int64_t kap_stride;
  Rhs rhs;
  Arenas arenas;
  int32_t* status;
  int max_nf, max_m, max_b;
  int max_rect;             // leaves: vertices of the largest closed rectangle
  Profiler* prof;            // nullptr unless profiling
  double fl_chol, fl_trsm, fl_syrk, fl_rhs;   // algorithmic flops of this launch (whole batch)
  uint32_t wait_limit;       // polls of a bounded mbarrier wait before it gives up
  int stall_node, stall_sample;   // test hook of the bounded waits (-1: off)
  // launches over several plans: the nodes and maps are the plans' tables
  // concatenated, plan_of[node] names the node's plan and plans[] its part (null
  // for a single plan)
  const PlanDev* plans;
  const int32_t* plan_of;
};

// Take the per-plan fields of `a` from the node's plan (no-op for one plan).  After
// it, a.batch is that plan's batch: CTAs of samples beyond it have no work.
__device__ __forceinline__ void bind_plan(StepArgs& a, int node) {
  if (!a.plan_of) return;
  const PlanDev& P = a.plans[a.plan_of[node]];
  a.arenas = P.arenas;
  a.kappa = P.kappa;
  a.kappa32 = P.kappa32;
  a.kap_stride = P.kap_stride;
  a.status = P.status;
  a.rhs = P.rhs;
  a.N = P.N;
  a.batch = P.batch;
}

// Fused bottom subtrees of the upsweep (one CTA per subtree and sample)
struct FuseArgs {
  StepArgs a;
  const int32_t* roots;       // [nroots x 12] subtree descriptors
  const int32_t* fused;       // node lists, bottom-up
  const int32_t* fuse_soff;   // per node: offset of its Schur square in the level buffer
  int sbuf_elems;             // elements of one level buffer
  int front_elems;            // elements of the front workspace shared by the warp groups
};
template <typename T> cudaError_t launch_subtree(const FuseArgs& f, int nroots, size_t smem_bytes, cudaStream_t st);

// mean functionals of the subdomains (Sec. 5.1 Lemma, Sec. 5.2): lambda^g of every node in
// the list (to the node's Schur slot, and to lam for observed nodes) and mu^f = (lambda^f, c)
struct FuncArgs {
  const NodeDev* nodes;
  const int32_t* maps;
  const int32_t* list;
  int nlist;
  int batch;
  int N;
  Arenas A;
  double* fmu;              // [batch x n_nodes]
  int64_t n_nodes;
  double* lam;              // [batch x lam_stride]: lambda^g of the observed nodes
  int64_t lam_stride;
  const int32_t* lam_off;   // per node, offset into a sample's lam row, or -1
};
template <typename T> cudaError_t launch_func_leaf(const FuncArgs& f, cudaStream_t st);
template <typename T> cudaError_t launch_func_warp(const FuncArgs& f, int max_nf, cudaStream_t st);
// observation k = mean over obs_nodes[k]: (lambda^g, x on its boundary) + mu^f (+ base)
cudaError_t launch_mean_obs(const FuncArgs& f, const int32_t* obs_nodes, int n_obs, const double* x,
                            int64_t x_stride, const double* base, double* u_obs, cudaStream_t st);

// warps per front of the grouped front kernel for a list's largest front (k_group.cu)
int group_warps(int max_nf, bool fp64);
// one upsweep list (api.cu): its sizes on the arguments, its launch(es), their count
void set_list(StepArgs& a, const ListInfo& li, double scale);
cudaError_t launch_step(int kind, StepArgs& a, cudaStream_t st);
int step_launches(int kind, const ListInfo& li);
// a plan's workspace as one part of a launch over several plans (api.cu)
PlanDev plan_part(const Plan& p, int batch, void* ws);

// many loads and Dirichlet data through the stored factors (k_data.cu): groups of
// kData right-hand sides share each factor read
constexpr int kData = 4;
struct DataArgs {
  const NodeDev* nodes;
  const int32_t* maps;
  Arenas A;
  int N, batch, n_loads;
  int nk;                 // loads of the current group (<= kData)
  double h2;              // h^2: vertex-quadrature weight of a nodal load on this mesh
  double* u;              // [batch x n_loads x N^2] the solutions (Dirichlet data at the boundary)
  double* d;              // [kData x batch x N^2] y_g during the sweep, then the correction
  double* r;              // [kData x batch x N^2] residuals of the group
  double* conv;           // [batch x 4] refinement bookkeeping
  int32_t* status;        // [batch] per-sample status words
};
cudaError_t launch_data_init(const DataArgs& D, const double* g, int k0, cudaStream_t st);
cudaError_t launch_data_residual(const DataArgs& D, const double* kappa, int64_t kap_stride, const double* c,
                                 const double* fH, int k0, cudaStream_t st);
template <typename T>
cudaError_t launch_data_sweep(const DataArgs& D, const int32_t* list, int nlist, int max_nf, int max_m, bool descent,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_data_leaf(const DataArgs& D, const int32_t* list, int nlist, bool descent, cudaStream_t st);
cudaError_t launch_data_update(const DataArgs& D, int k0, double tol, bool last, bool test, cudaStream_t st);

// assembly: kappa = exp(Phi Z) (Sec. 3.1; kappa = e^q)
cudaError_t launch_kappa(const double* phi, const double* Z, int n_t, int n_z, int batch, double* kappa,
                         float* kappa32, int64_t kap_stride, cudaStream_t st);
// the same in double-float arithmetic (mixed plans; Phi pre-split into FP32 hi + lo)
cudaError_t launch_kappa_df(const float* phi_hi, const float* phi_lo, const double* Z, int n_t, int n_z, int batch,
                            double* kappa, float* kappa32, int64_t kap_stride, cudaStream_t st);

// sweeps with one warp per (node, sample)
template <typename T>
cudaError_t launch_forward_warp(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, int max_nf, int max_m, cudaStream_t st);
template <typename T>
cudaError_t launch_descent_warp(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, int max_nf, int max_m,
                                cudaStream_t st);
// right-hand-side sweep over fronts of 16..32 eliminated vertices and at most 256 rows,
// rows in registers
constexpr int kMidMaxRows = 256;
template <typename T>
cudaError_t launch_forward_mid(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                               const Arenas& A, const Rhs& rhs, cudaStream_t st);
// sweeps over fronts of at most 32 rows, factor rows in registers
template <typename T>
cudaError_t launch_forward_tiny(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, cudaStream_t st);
template <typename T>
cudaError_t launch_descent_tiny(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, cudaStream_t st);
// fronts of up to kSmallMax rows: W warps per front, several samples of a node per CTA
template <typename T> cudaError_t launch_front_group(const StepArgs& a, int family, cudaStream_t st);
// condensed leaves (K_gg^-1 and boundary couplings): upsweep, right-hand-side sweep, descent
template <typename T> cudaError_t launch_leaf_front(const StepArgs& a, cudaStream_t st);
template <typename T>
cudaError_t launch_leaf_forward(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, cudaStream_t st);
template <typename T>
cudaError_t launch_leaf_descent(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, cudaStream_t st);
// SYRK of large FP32 fronts on the tensor cores (tcgen05, 3xTF32)
cudaError_t launch_syrk_tc(const StepArgs& a, cudaStream_t st);
// large fronts: fill in global memory, then POTRF of gamma, TRSM of the rest, SYRK into S
template <typename T> cudaError_t launch_front_large(const StepArgs& a, cudaStream_t st);

// sweeps over the fused bottom subtrees (k_sweep.cu): one warp per (subtree, sample)
struct SubArgs {
  const NodeDev* nodes;
  const int32_t* maps;
  const int32_t* subs;     // [n_sub x kSubInts]
  const int32_t* sched;    // [nodes x kSchedInts], pre-order per subtree
  const int16_t* rec;      // map records
  Arenas A;
  int N, batch;
  // per warp: the subtree's factor range, y_g range (descent), rectangle, stack (sweep)
  int fac_bytes, y_bytes, region_bytes, stack_bytes, warp_bytes;
  int sched_bytes, rec_bytes;                  // per CTA
};
template <typename T>
cudaError_t launch_descent_sub(const SubArgs& g, int n_sub, size_t smem, double* u, int64_t u_stride,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_forward_sub(const SubArgs& g, int n_sub, size_t smem, const Rhs& rhs, cudaStream_t st);

// descent (Root to Leaves) over a list of nodes of one depth; u is FP64 [batch x N^2]
template <typename T>
cudaError_t launch_descent(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                           const Arenas& A, double* u, int64_t u_stride, int max_b, int max_m, cudaStream_t st);

// iterative refinement (mixed precision)
template <typename T>
cudaError_t launch_forward(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                           const Arenas& A, const Rhs& rhs, int max_nf, cudaStream_t st);
// r = b - A u with b = load (loadv == nullptr) or the vertex vector loadv
cudaError_t launch_residual(const double* kappa, int64_t kap_stride, const double* u, int64_t u_stride, int N,
                            double load, const double* loadv, int64_t load_stride, double* r, int64_t r_stride,
                            int batch, cudaStream_t st);
cudaError_t launch_update(double* u, int64_t u_stride, const double* du, int64_t du_stride, int N, int batch,
                          cudaStream_t st);
// refinement of full-field solves: correction size over every unknown, convergence test at the last step
cudaError_t launch_conv_full(const double* du, int64_t du_stride, const double* u, int64_t u_stride, int N,
                             double tol, double* dprev, int32_t* status, bool last, int batch, cudaStream_t st);
// subdomain means (Sec. 5, Eq. mean): leaves from u, fathers from their sons
cudaError_t launch_leaf_means(const NodeDev* nodes, const int32_t* list, int n, const double* u, int64_t u_stride,
                              int N, double* means, int64_t m_stride, int batch, cudaStream_t st);
cudaError_t launch_father_means(const NodeDev* nodes, const int32_t* list, int n, double* means, int64_t m_stride,
                                int batch, cudaStream_t st);
cudaError_t launch_delta_obs(const double* du, int64_t stride, const int32_t* obs, int n_obs, double* dprev,
                             int batch, cudaStream_t st);
cudaError_t launch_final_obs(const double* u, const double* du, int64_t stride, const int32_t* obs, int n_obs,
                             double tol, const double* dprev, double* u_obs, int32_t* status, int batch,
                             cudaStream_t st);

cudaError_t launch_gather_obs(const double* u, int64_t u_stride, const int32_t* obs, int n_obs, int batch,
                              double* u_obs, cudaStream_t st);
cudaError_t launch_loglik(const double* u_obs, int n_obs, int batch, const double* y, int y_per_sample, double sigma,
                          const int32_t* status, double* loglik, cudaStream_t st);

}  // namespace hdd
