// Iterative refinement of the mixed-precision path: FP64 residual of the global
// FE system, a right-hand-side-only sweep through the stored factors, update.
//
// With factors L (the partial Cholesky factors of every node, FP32 below the
// top levels) the HDD solve of A x = r is: leaves to root, z_g = sum of the sons'
// condensed right-hand sides + r_g, y_g = L_gg^-1 z_g, condensed z_B - L_Bg y_g
// (the bordered row of the upsweep, Eq. SchurC1 applied to a new F c); then the
// unchanged descent (Root to Leaves).  The residual r = b - A u uses the FP64
// stiffness of Eq. coefA (5-point edge weights of the "/" mesh) and the FP64 u.
#include "launch.h"

namespace hdd {

template <typename T> __device__ __forceinline__ T* fwd_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* fwd_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* fwd_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* fwd_S(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* fwd_S<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* fwd_S<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

// condensed right-hand side entry p of a son, stored contiguously at the start
// of the son's Schur block by the son's own right-hand-side sweep
__device__ __forceinline__ double son_rhs(const Arenas& A, const NodeDev& ch, int s, int p) {
  const int64_t idx = (int64_t)p + ch.s_off;
  return ch.fp64 ? A.s64[(int64_t)s * A.s64_stride + idx] : (double)A.s32[(int64_t)s * A.s32_stride + idx];
}

// Right-hand-side sweep at one node: one CTA per (node, sample).  Forward
// substitution with L_gg in 32-column blocks (one warp, shuffles), each block
// folded into every row below it (one thread per row, coalesced down columns).
template <typename T>
__global__ void k_forward(const NodeDev* __restrict__ nodes, const int32_t* __restrict__ maps,
                          const int32_t* __restrict__ list, Arenas A, Rhs rhs) {
  const int node = list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  T* F = fwd_F<T>(A, nd, s);
  const int32_t* vid = maps + nd.map_off;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw);   // [nf - 1]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nd.leaf) {
    for (int r = threadIdx.x; r < nf - 1; r += blockDim.x) z[r] = (r < m) ? (T)rhs(s, vid[r]) : (T)0;
  } else {
    const NodeDev c0 = nodes[nd.child0], c1 = nodes[nd.child1];
    const int32_t* pos0 = vid + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    for (int r = threadIdx.x; r < nf - 1; r += blockDim.x) {
      T v = (r < m) ? (T)rhs(s, vid[r]) : (T)0;
      if (pos0[r] >= 0) v += (T)son_rhs(A, c0, s, pos0[r]);
      if (pos1[r] >= 0) v += (T)son_rhs(A, c1, s, pos1[r]);
      z[r] = v;
    }
  }
  T* Ld = z + ((nf + 3) & ~3);   // [32][33] diagonal block of L_gg, staged per block
  // the next block's diagonal block is loaded into registers (four entries per thread)
  // while the current block is solved and folded
  T dpre[4];
  auto fetch_diag = [&](int cb) {
    const int jb = min(32, m - cb);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int idx = threadIdx.x + k * 256, c = idx >> 5, l = idx & 31;
      dpre[k] = (c < jb && l < jb) ? F[(int64_t)(cb + c) * nf + cb + l] : (T)0;
    }
  };
  if (m > 0) fetch_diag(0);
  for (int cb = 0; cb < m; cb += 32) {
    const int jb = min(32, m - cb);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int idx = threadIdx.x + k * 256;
      Ld[(idx >> 5) * 33 + (idx & 31)] = dpre[k];
    }
    __syncthreads();
    if (cb + 32 < m) fetch_diag(cb + 32);
    if (warp == 0) {
      T x = (lane < jb) ? z[cb + lane] : (T)0;
      for (int c = 0; c < jb; ++c) {
        T yc = __shfl_sync(0xffffffffu, x, c);
        yc = yc / Ld[c * 33 + c];
        if (lane == c) x = yc;
        if (lane > c && lane < jb) x -= Ld[c * 33 + lane] * yc;
      }
      if (lane < jb) z[cb + lane] = x;
    }
    __syncthreads();
    for (int i = cb + jb + threadIdx.x; i < nf - 1; i += blockDim.x) {
      T acc = (T)0;
      if (jb == 32) {   // the block's 32 entries of row i, all loads in flight first
        T f[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) f[c] = F[(int64_t)(cb + c) * nf + i];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc += f[c] * z[cb + c];
      } else {
        for (int c = 0; c < jb; ++c) acc += F[(int64_t)(cb + c) * nf + i] * z[cb + c];
      }
      z[i] -= acc;
    }
  }
  __syncthreads();
  T* Y = node_Y<T>(A, nd, s);
  for (int c = threadIdx.x; c < m; c += blockDim.x) Y[c] = z[c];
  if (b > 0) {
    T* S = fwd_S<T>(A, nd, s);
    for (int r = threadIdx.x; r < b; r += blockDim.x) S[r] = z[m + r];
  }
}

template <typename T>
cudaError_t launch_forward(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                           const Arenas& A, const Rhs& rhs, int max_nf, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  const size_t smem = ((size_t)((max_nf + 3) & ~3) + 32 * 33) * sizeof(T);
  k_forward<T><<<dim3(nlist, batch), 256, smem, st>>>(nodes, maps, list, A, rhs);
  return cudaGetLastError();
}
template cudaError_t launch_forward<double>(const NodeDev*, const int32_t*, const int32_t*, int, int, const Arenas&,
                                            const Rhs&, int, cudaStream_t);
template cudaError_t launch_forward<float>(const NodeDev*, const int32_t*, const int32_t*, int, int, const Arenas&,
                                           const Rhs&, int, cudaStream_t);

// r = b - A u over the unknowns (FP64).  (A u)_v = sum over the four axis edges of
// w_e (u_v - u_w), w_e = mean kappa of the two triangles having e as a leg;
// Dirichlet neighbours contribute u_w = 0.  Boundary entries of r are set to 0.
// b is the constant vertex load `load`, or the vector loadv [batch x load_stride]
// when it is not null.
// A thread owns one column i of vertices over kResRows consecutive rows and
// slides up them, so that every row of u and of the cells' kappa is loaded once
// per thread (the right neighbour comes from the adjacent thread's loads through
// L1, the left one's edge terms by a shuffle).
constexpr int kResRows = 8;

__global__ void __launch_bounds__(128) k_residual(const double* __restrict__ kappa, int64_t kap_stride,
                                                  const double* __restrict__ u, int64_t u_stride, int N,
                                                  double load, const double* __restrict__ loadv,
                                                  int64_t load_stride, double* __restrict__ r, int64_t r_stride) {
  const int s = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * kResRows;
  const bool live = i < N;   // every lane stays for the shuffles
  const double* ks = kappa + (int64_t)s * kap_stride;
  const double* us = u + (int64_t)s * u_stride;
  double* rs = r + (int64_t)s * r_stride;
  const double* bs = loadv ? loadv + (int64_t)s * load_stride : nullptr;
  const bool col_in = i >= 1 && i <= N - 2;
  auto urow = [&](int j, int di) {   // u at (i + di, j), 0 off the unknowns
    const int ii = i + di;
    return (ii >= 1 && ii <= N - 2 && j >= 1 && j <= N - 2) ? us[(int64_t)j * N + ii] : 0.0;
  };
  // kappa of the lower-right (t = 0) and upper-left (t = 1) triangles of cells (i, j) and (i - 1, j)
  auto kc = [&](int ci, int j, int t) {
    return (ci >= 0 && ci <= N - 2 && j >= 0 && j <= N - 2) ? ks[2 * ((int64_t)j * (N - 1) + ci) + t] : 0.0;
  };
  // Each edge's weight sum (twice its weight) and the difference of u along it are
  // formed once: a thread forms those of its east and north edges; its west edge is
  // the east edge of the lane to its left (a shuffle; lane 0 forms it itself), its
  // south edge the north edge of the row below (carried).  Au = sum over the four
  // edges of (weight sum) x (difference) / 2, and r = b - Au is one FMA.
  double u_c = live ? urow(j0, 0) : 0.0;
  double kb0 = live ? kc(i, j0 - 1, 1) : 0.0;                  // upper-left of (i, j-1)
  double sum_d = live ? kb0 + kc(i - 1, j0 - 1, 0) : 0.0;      // edge (i, j-1)-(i, j)
  double d_s = live ? u_c - urow(j0 - 1, 0) : 0.0;             // u_c - u south
  for (int j = j0; j < min(j0 + kResRows, N); ++j) {
    double u_n = 0.0, ue = 0.0, ka0 = 0.0, ka1 = 0.0, ka2 = 0.0;
    if (live) {
      u_n = urow(j + 1, 0);
      ue = urow(j, 1);
      ka0 = kc(i, j, 0);
      ka1 = kc(i, j, 1);
      ka2 = kc(i - 1, j, 0);
    }
    const double sum_r = ka0 + kb0;   // edge (i, j)-(i+1, j): lower-right of (i, j), upper-left of (i, j-1)
    const double sum_u = ka1 + ka2;   // edge (i, j)-(i, j+1): upper-left of (i, j), lower-right of (i-1, j)
    const double d_e = u_c - ue, d_n = u_c - u_n;
    // west edge: the left neighbour's east edge, with the difference's sign turned
    double sum_l = __shfl_up_sync(0xffffffffu, sum_r, 1);
    double d_w = -__shfl_up_sync(0xffffffffu, d_e, 1);
    if (lane == 0 && live) {
      sum_l = ka2 + kc(i - 1, j - 1, 1);   // lower-right of (i-1, j), upper-left of (i-1, j-1)
      d_w = u_c - urow(j, -1);
    }
    if (live) {
      if (!col_in || j < 1 || j > N - 2) {
        rs[(int64_t)j * N + i] = 0.0;
      } else {
        const double Au2 = sum_r * d_e + sum_l * d_w + sum_u * d_n + sum_d * d_s;
        rs[(int64_t)j * N + i] = fma(-0.5, Au2, bs ? bs[(int64_t)j * N + i] : load);
      }
    }
    sum_d = sum_u;
    d_s = -d_n;
    u_c = u_n;
    kb0 = ka1;
  }
}

cudaError_t launch_residual(const double* kappa, int64_t kap_stride, const double* u, int64_t u_stride, int N,
                            double load, const double* loadv, int64_t load_stride, double* r, int64_t r_stride,
                            int batch, cudaStream_t st) {
  k_residual<<<dim3((N + 127) / 128, (N + kResRows - 1) / kResRows, batch), 128, 0, st>>>(
      kappa, kap_stride, u, u_stride, N, load, loadv, load_stride, r, r_stride);
  return cudaGetLastError();
}

// u += du at every interior vertex
__global__ void k_update(double* __restrict__ u, int64_t u_stride, const double* __restrict__ du,
                         int64_t du_stride, int N) {
  const int s = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N * N) return;
  const int i = v % N, j = v / N;
  if (i < 1 || j < 1 || i > N - 2 || j > N - 2) return;
  u[(int64_t)s * u_stride + v] += du[(int64_t)s * du_stride + v];
}

cudaError_t launch_update(double* u, int64_t u_stride, const double* du, int64_t du_stride, int N, int batch,
                          cudaStream_t st) {
  const int NN = N * N;
  k_update<<<dim3((NN + 255) / 256, batch), 256, 0, st>>>(u, u_stride, du, du_stride, N);
  return cudaGetLastError();
}

// Size of a refinement correction over every unknown (full-field solves):
// d = max_v |du_v| per sample.  Before the last step d is kept in dprev; after
// the last update the remaining error, estimated as d_K min(1, d_K / d_{K-1})
// (no contraction credit when d_{K-1} = 0), is compared with tol * max_v |u_v|
// and a sample above it is marked HDD_ENOCONV.
constexpr int kConvThreads = 512;
__global__ void __launch_bounds__(kConvThreads) k_conv_full(const double* __restrict__ du, int64_t du_stride,
                                                           const double* __restrict__ u, int64_t u_stride, int N,
                                                           double tol, double* __restrict__ dprev,
                                                           int32_t* status, int last) {
  __shared__ double red_d[kConvThreads], red_u[kConvThreads];
  const int s = blockIdx.x;
  const int n = N - 2;   // unknowns per row and column
  double md = 0.0, mu = 0.0;
  for (int q = threadIdx.x; q < n * n; q += kConvThreads) {
    const int64_t v = (int64_t)(q / n + 1) * N + (q % n + 1);
    md = fmax(md, fabs(du[(int64_t)s * du_stride + v]));
    if (last) mu = fmax(mu, fabs(u[(int64_t)s * u_stride + v]));
  }
  red_d[threadIdx.x] = md;
  red_u[threadIdx.x] = mu;
  __syncthreads();
  for (int w = kConvThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red_d[threadIdx.x] = fmax(red_d[threadIdx.x], red_d[threadIdx.x + w]);
      red_u[threadIdx.x] = fmax(red_u[threadIdx.x], red_u[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double dK = red_d[0];
  if (!last) {
    dprev[s] = dK;
    return;
  }
  const double dp = dprev[s];
  const double est = (dp > 0.0) ? dK * fmin(1.0, dK / dp) : dK;
  if (tol >= 0.0 && !(est <= tol * red_u[0])) flag_status(status, s, -HDD_ENOCONV, 0);
}

cudaError_t launch_conv_full(const double* du, int64_t du_stride, const double* u, int64_t u_stride, int N,
                             double tol, double* dprev, int32_t* status, bool last, int batch, cudaStream_t st) {
  k_conv_full<<<batch, kConvThreads, 0, st>>>(du, du_stride, u, u_stride, N, tol, dprev, status, last ? 1 : 0);
  return cudaGetLastError();
}

// max_k |du[obs_k]| per sample (the size of a refinement correction), kept for
// the contraction estimate of the last step.
__global__ void k_delta_obs(const double* __restrict__ du, int64_t stride, const int32_t* __restrict__ obs,
                            int n_obs, double* __restrict__ dprev) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  double md = 0.0;
  for (int k = threadIdx.x; k < n_obs; k += blockDim.x) md = fmax(md, fabs(du[(int64_t)s * stride + obs[k]]));
  red[threadIdx.x] = md;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) dprev[s] = red[0];
}

cudaError_t launch_delta_obs(const double* du, int64_t stride, const int32_t* obs, int n_obs, double* dprev,
                             int batch, cudaStream_t st) {
  k_delta_obs<<<batch, 256, 0, st>>>(du, stride, obs, n_obs, dprev);
  return cudaGetLastError();
}

// Last refinement step: u_obs = u[obs] + du[obs].  The error left after this
// update is estimated from the observed contraction, d_K * min(1, d_K / d_{K-1})
// with d = max_k |du_k| (d_{K-1} = 0, i.e. no contraction credit, after a single
// step); a sample whose estimate exceeds tol * max_k |u_obs_k| is marked HDD_ENOCONV.
__global__ void k_final_obs(const double* __restrict__ u, const double* __restrict__ du, int64_t stride,
                            const int32_t* __restrict__ obs, int n_obs, double tol, const double* __restrict__ dprev,
                            double* __restrict__ u_obs, int32_t* status) {
  __shared__ double red_d[256], red_u[256];
  const int s = blockIdx.x;
  double md = 0.0, mu = 0.0;
  for (int k = threadIdx.x; k < n_obs; k += blockDim.x) {
    const double d = du ? du[(int64_t)s * stride + obs[k]] : 0.0;
    const double v = u[(int64_t)s * stride + obs[k]] + d;
    u_obs[(int64_t)s * n_obs + k] = v;
    md = fmax(md, fabs(d));
    mu = fmax(mu, fabs(v));
  }
  red_d[threadIdx.x] = md;
  red_u[threadIdx.x] = mu;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red_d[threadIdx.x] = fmax(red_d[threadIdx.x], red_d[threadIdx.x + w]);
      red_u[threadIdx.x] = fmax(red_u[threadIdx.x], red_u[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && tol >= 0.0) {
    const double dK = red_d[0], dp = dprev ? dprev[s] : 0.0;
    const double est = (dp > 0.0) ? dK * fmin(1.0, dK / dp) : dK;
    if (!(est <= tol * red_u[0])) flag_status(status, s, -HDD_ENOCONV, 0);
  }
}

cudaError_t launch_final_obs(const double* u, const double* du, int64_t stride, const int32_t* obs, int n_obs,
                             double tol, const double* dprev, double* u_obs, int32_t* status, int batch,
                             cudaStream_t st) {
  k_final_obs<<<batch, 256, 0, st>>>(u, du, stride, obs, n_obs, tol, dprev, u_obs, status);
  return cudaGetLastError();
}

cudaError_t configure_refine_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_forward<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_forward<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
