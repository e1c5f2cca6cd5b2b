// Mean values of the solution over subdomains of the tree without the full
// solution (Sec. 5, Eq. mean; Sec. 5.1 Lemma, Eq. prop1 / prop2; the two
// algorithms of Sec. 5.2 that build lambda^g and lambda^f).
//
// The mean over omega is a linear functional of the data of omega,
//   mean(omega) = (lambda^g_omega, u on the boundary unknowns of omega)
//               + (lambda^f_omega, load at the unknowns inside omega),
// and a father's vectors follow from its sons' with c_i = |omega_i| / |omega|:
//   z          = c_1 lambda^g_1 + c_2 lambda^g_2   extended to the father front [gamma, B]
//   lambda^g   = z_B + (Phi^g)^T z_gamma,   lambda^f = sum_i c_i lambda^f_i| + (Phi^f)^T z_gamma.
// With the stored partial Cholesky factors, Phi^g = -L_gg^-T L_Bg^T and
// Phi^f c = L_gg^-T y_g (y_g = L_gg^-1 times the condensed load on gamma), so
//   w = L_gg^-1 z_gamma,   lambda^g = z_B - L_Bg w,   (lambda^f, c) = sum_i c_i (lambda^f_i, c_i) + w . y_g:
// the transposed-Phi products are a right-hand-side sweep through the factors
// with the sons' vectors, weighted by c_i, as the right-hand side.  Only the
// scalar mu^f = (lambda^f, c) for the load c of the factorisation is kept (the
// load enters through the stored y_g), never the vector lambda^f.
//
// Leaves start from the definition of the mean over their own triangles: the
// weight of vertex v is the summed |t|/3 of the leaf's triangles at v (h^2/6 per
// triangle), divided by |omega|; the paper's triangle leaves start from
// (1/3, 1/3, 1/3), which is the same rule for one triangle.
#include "launch.h"

namespace hdd {

namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kLeafSamples = 16;   // condensed leaves: one half-warp per sample
constexpr int kFuncWarps = 8;      // other nodes: one warp per sample, 8 samples of a node per CTA

// Eq. mean over the rectangle of nd: weight of vertex v divided by |omega|.
// Vertex (i, j) touches both triangles of cells (i, j) and (i-1, j-1), the
// lower-right one of cell (i-1, j) and the upper-left one of cell (i, j-1).
__device__ __forceinline__ double mean_weight(int v, int N, const NodeDev& nd) {
  const int vi = v % N, vj = v / N;
  auto in = [&](int ci, int cj) { return ci >= nd.x0 && ci < nd.x1 && cj >= nd.y0 && cj < nd.y1; };
  const int cnt = (in(vi, vj) ? 2 : 0) + (in(vi - 1, vj) ? 1 : 0) + (in(vi - 1, vj - 1) ? 2 : 0) +
                  (in(vi, vj - 1) ? 1 : 0);
  return cnt / (6.0 * (double)(nd.x1 - nd.x0) * (double)(nd.y1 - nd.y0));
}

__device__ __forceinline__ double area(const NodeDev& nd) { return (double)(nd.x1 - nd.x0) * (double)(nd.y1 - nd.y0); }

template <typename T> __device__ __forceinline__ const T* fn_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ const double* fn_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ const float* fn_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
// lambda^g of a node is handed to its father at the start of the node's (unused)
// Schur block, in the node's precision, as the right-hand-side sweep does
template <typename T> __device__ __forceinline__ T* fn_slot(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* fn_slot<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* fn_slot<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}
__device__ __forceinline__ double son_lambda(const Arenas& A, const NodeDev& ch, int s, int p) {
  const int64_t idx = (int64_t)p + ch.s_off;
  return ch.fp64 ? A.s64[(int64_t)s * A.s64_stride + idx] : (double)A.s32[(int64_t)s * A.s32_stride + idx];
}

// packed lower column-major index of (i, j), i >= j, of an m x m matrix (condensed leaves' G)
__device__ __forceinline__ int pk(int i, int j, int m) { return j * m - j * (j - 1) / 2 + (i - j); }

}  // namespace

// Condensed leaves (G = K_gg^-1 and one coupling weight w_i = K_Bg[i, c_i] per
// boundary row): lambda^f = G w_I, lambda^g_i = w_B,i - w_i (G w_I)[c_i], and
// mu^f = (G w_I) . c_I = w_I . (G c_I) = w_I . y_g.  One half-warp per (leaf, sample).
template <typename T>
__global__ void __launch_bounds__(256) k_func_leaf(FuncArgs f) {
  const int node = f.list[blockIdx.x];
  const int hw = threadIdx.x >> 4, r = threadIdx.x & 15;
  const int s = blockIdx.y * kLeafSamples + hw;
  const bool active = s < f.batch;   // both half-warps stay for the shuffles
  const int ss = active ? s : 0;
  const NodeDev nd = f.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = f.maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const T* G = fn_F<T>(f.A, nd, ss);
  const double wr = (r < m) ? mean_weight(vid[r], f.N, nd) : 0.0;
  T v = (T)0;
#pragma unroll
  for (int j = 0; j < kLeafInvMax; ++j) {
    const T wj = __shfl_sync(kAll, (T)wr, j, 16);
    if (r < m && j < m) v += G[r >= j ? pk(r, j, m) : pk(j, r, m)] * wj;
  }
  double mu = (r < m) ? wr * (double)node_Y<T>(f.A, nd, ss)[r] : 0.0;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) mu += __shfl_xor_sync(kAll, mu, o, 16);
  if (active && r == 0) f.fmu[(int64_t)s * f.n_nodes + node] = mu;
  T* slot = fn_slot<T>(f.A, nd, ss);
  const int off = f.lam_off[node];
  const int g_elems = m * (m + 1) / 2;
  for (int i0 = 0; i0 < b; i0 += 16) {
    const int i = i0 + r;
    const int ci = (i < b) ? cpl[i] : -1;
    const T vc = __shfl_sync(kAll, v, ci >= 0 ? ci : 0, 16);
    if (active && i < b) {
      T lg = (T)mean_weight(vid[m + i], f.N, nd);
      if (ci >= 0) lg -= G[g_elems + i] * vc;
      slot[i] = lg;
      if (off >= 0) f.lam[(int64_t)s * f.lam_stride + off + i] = (double)lg;
    }
  }
}

// Every other node (leaves with partial Cholesky factors, fathers): one warp per
// (node, sample).  z over the front rows [gamma, B]: a leaf's mean weights, or
// the sons' lambda^g weighted by c_i and added through the extend-add maps
// (Sec. 3.3, Eq. block_equation4, positions pos0 / pos1); then forward
// substitution with L_gg, folding each column into the rows below it, which
// leaves w = L_gg^-1 z_gamma in the gamma rows and z_B - L_Bg w in the boundary
// rows (lambda^g); mu^f = c_1 mu_1 + c_2 mu_2 + w . y_g.
template <typename T>
__global__ void __launch_bounds__(32 * kFuncWarps) k_func_warp(FuncArgs f, int wstride) {
  const int node = f.list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * kFuncWarps + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw) + warp * wstride;
  if (s >= f.batch) return;
  const NodeDev nd = f.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = f.maps + nd.map_off;
  const T* F = fn_F<T>(f.A, nd, s);
  double mu = 0.0;
  if (nd.leaf) {
    for (int r = lane; r < nf - 1; r += 32) z[r] = (T)mean_weight(vid[r], f.N, nd);
  } else {
    const NodeDev c0 = f.nodes[nd.child0], c1 = f.nodes[nd.child1];
    const double a = area(nd), w0 = area(c0) / a, w1 = area(c1) / a;
    const int32_t* pos0 = vid + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    for (int r = lane; r < nf - 1; r += 32) {
      double val = 0.0;
      const int q0 = pos0[r], q1 = pos1[r];
      if (q0 >= 0) val += w0 * son_lambda(f.A, c0, s, q0);
      if (q1 >= 0) val += w1 * son_lambda(f.A, c1, s, q1);
      z[r] = (T)val;
    }
    if (lane == 0)
      mu = w0 * f.fmu[(int64_t)s * f.n_nodes + nd.child0] + w1 * f.fmu[(int64_t)s * f.n_nodes + nd.child1];
  }
  __syncwarp();
  for (int c = 0; c < m; ++c) {
    const T* col = F + (int64_t)c * nf;
    const T wc = z[c] / col[c];
    for (int i = c + 1 + lane; i < nf - 1; i += 32) z[i] -= col[i] * wc;
    __syncwarp();
    if (lane == 0) z[c] = wc;
    __syncwarp();
  }
  const T* Y = node_Y<T>(f.A, nd, s);
  double acc = 0.0;
  for (int c = lane; c < m; c += 32) acc += (double)z[c] * (double)Y[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
  if (lane == 0) f.fmu[(int64_t)s * f.n_nodes + node] = mu + acc;
  if (b > 0) {
    T* slot = fn_slot<T>(f.A, nd, s);
    const int off = f.lam_off[node];
    for (int r = lane; r < b; r += 32) {
      const T lg = z[m + r];
      slot[r] = lg;
      if (off >= 0) f.lam[(int64_t)s * f.lam_stride + off + r] = (double)lg;
    }
  }
}

// Observation k of sample s: the mean over node obs_nodes[k] by Eq. prop1,
//   (lambda^g, x on the node's boundary unknowns) + mu^f (+ base[node]),
// with x = u (the descent to the node's ancestors) or, on refined mixed plans, x =
// the last correction and base = the means of the refined iterate.  One warp per
// (observation, sample).
__global__ void __launch_bounds__(256) k_mean_obs(FuncArgs f, const int32_t* __restrict__ obs_nodes, int n_obs,
                                                  const double* __restrict__ x, int64_t x_stride,
                                                  const double* __restrict__ base, double* __restrict__ u_obs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + warp;
  const int s = blockIdx.y;
  if (k >= n_obs) return;
  const int node = obs_nodes[k];
  const NodeDev nd = f.nodes[node];
  const int32_t* bnd = f.maps + nd.map_off + nd.m;
  const double* lam = f.lam + (int64_t)s * f.lam_stride + f.lam_off[node];
  const double* xs = x + (int64_t)s * x_stride;
  double acc = 0.0;
  for (int i = lane; i < nd.b; i += 32) acc += lam[i] * xs[bnd[i]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kAll, acc, o);
  if (lane == 0) {
    double v = acc + f.fmu[(int64_t)s * f.n_nodes + node];
    if (base) v += base[(int64_t)s * f.n_nodes + node];
    u_obs[(int64_t)s * n_obs + k] = v;
  }
}

template <typename T>
cudaError_t launch_func_leaf(const FuncArgs& f, cudaStream_t st) {
  if (f.nlist == 0) return cudaSuccess;
  k_func_leaf<T><<<dim3(f.nlist, (f.batch + kLeafSamples - 1) / kLeafSamples), 256, 0, st>>>(f);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_func_warp(const FuncArgs& f, int max_nf, cudaStream_t st) {
  if (f.nlist == 0) return cudaSuccess;
  const int ws = (max_nf + 3) & ~3;
  const size_t smem = (size_t)kFuncWarps * ws * sizeof(T);
  k_func_warp<T><<<dim3(f.nlist, (f.batch + kFuncWarps - 1) / kFuncWarps), 32 * kFuncWarps, smem, st>>>(f, ws);
  return cudaGetLastError();
}

cudaError_t launch_mean_obs(const FuncArgs& f, const int32_t* obs_nodes, int n_obs, const double* x,
                            int64_t x_stride, const double* base, double* u_obs, cudaStream_t st) {
  k_mean_obs<<<dim3((n_obs + 7) / 8, f.batch), 256, 0, st>>>(f, obs_nodes, n_obs, x, x_stride, base, u_obs);
  return cudaGetLastError();
}

template cudaError_t launch_func_leaf<double>(const FuncArgs&, cudaStream_t);
template cudaError_t launch_func_leaf<float>(const FuncArgs&, cudaStream_t);
template cudaError_t launch_func_warp<double>(const FuncArgs&, int, cudaStream_t);
template cudaError_t launch_func_warp<float>(const FuncArgs&, int, cudaStream_t);

cudaError_t configure_func_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_func_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_func_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
