// Many loads and Dirichlet data at a fixed coefficient field (Sec. 2: the node
// operators are computed once and applied to any number of right-hand sides and
// boundary data; Sec. 3.5: a right-hand side given on the coarse grid H = 2h).
//
// Every solve is written in correction form, u <- u + A_II^-1 (c - A u) with u
// holding the Dirichlet data g at the boundary vertices, so the boundary data,
// the load and (mixed plans) iterative refinement share one loop:
//   r = c - A u          the FP64 five-point residual of Eq. coefA; boundary
//                        neighbours contribute their g (first pass: c - A_IB g)
//   d = A_II^-1 r        "Leaves to Root" through the stored factors, then
//                        "Root to Leaves" over every node
//   u += d               at the interior vertices.
// Loads run in groups of kData right-hand sides: a warp (half-warp for condensed
// leaves) reads a node's factors once and applies them to every load of the
// group, so the factor traffic is shared by kData loads (a multi-right-hand-side
// sweep).  The group's y_g are kept in d at the node's gamma vertices (each
// unknown is eliminated by exactly one node) and its condensed right-hand sides
// at the start of the node's (unused) Schur block, load k at offset k * b
// (kData * b <= (b + 1)^2 for every b >= 1 when kData <= 4).
// A load on the coarse grid enters through its fine interpolant: the fine vertex
// (i, j) takes the coarse value at (i/2, j/2), or the mean of the two coarse ends
// of the coarse axis edge or "/" diagonal it halves; vertex quadrature makes the
// load h^2 times that value (Eq. coefc on this mesh).
#include "launch.h"

namespace hdd {

namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kDataWarps = 8;   // at most; fewer when the group's vectors of a large front need the room

template <typename T> __device__ __forceinline__ const T* dat_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ const double* dat_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ const float* dat_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* dat_slot(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* dat_slot<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* dat_slot<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}
__device__ __forceinline__ double son_cond(const Arenas& A, const NodeDev& ch, int s, int k, int p) {
  const int64_t idx = (int64_t)k * ch.b + p + ch.s_off;
  return ch.fp64 ? A.s64[(int64_t)s * A.s64_stride + idx] : (double)A.s32[(int64_t)s * A.s32_stride + idx];
}
__device__ __forceinline__ int pk(int i, int j, int m) { return j * m - j * (j - 1) / 2 + (i - j); }

}  // namespace

// u_k := g on the boundary vertices (0 without data), 0 inside; d_k := 0 (its
// boundary entries stay 0: the descent reads them as Dirichlet values of the correction).
__global__ void k_data_init(const DataArgs D, const double* __restrict__ g, int k0) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, k = blockIdx.z;
  const int N = D.N;
  if (v >= N * N) return;
  const int i = v % N, j = v / N;
  const bool bnd = i == 0 || j == 0 || i == N - 1 || j == N - 1;
  const int64_t o = ((int64_t)s * D.n_loads + k0 + k) * N * N + v;
  D.u[o] = (bnd && g) ? g[o] : 0.0;
  D.d[((int64_t)k * D.batch + s) * N * N + v] = 0.0;
}

// r_k = c_k - A u_k at the interior vertices (0 on the boundary); the load is the
// fine vector c or h^2 times the fine interpolant of the coarse nodal values f_H.
__global__ void __launch_bounds__(128) k_data_residual(const DataArgs D, const double* __restrict__ kappa,
                                                       int64_t kap_stride, const double* __restrict__ c,
                                                       const double* __restrict__ fH, int k0) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, k = blockIdx.z;
  const int N = D.N;
  if (v >= N * N) return;
  const int i = v % N, j = v / N;
  double* rs = D.r + ((int64_t)k * D.batch + s) * N * N;
  if (i < 1 || j < 1 || i > N - 2 || j > N - 2) {
    rs[v] = 0.0;
    return;
  }
  const int64_t lo = (int64_t)s * D.n_loads + k0 + k;
  const double* us = D.u + lo * N * N;
  const double* ks = kappa + (int64_t)s * kap_stride;
  auto kc = [&](int ci, int cj, int t) { return ks[2 * ((int64_t)cj * (N - 1) + ci) + t]; };
  // edge weights: mean kappa of the two triangles having the edge as a leg (Eq. coefA)
  const double wr = 0.5 * (kc(i, j, 0) + kc(i, j - 1, 1));
  const double wl = 0.5 * (kc(i - 1, j, 0) + kc(i - 1, j - 1, 1));
  const double wu = 0.5 * (kc(i, j, 1) + kc(i - 1, j, 0));
  const double wd = 0.5 * (kc(i, j - 1, 1) + kc(i - 1, j - 1, 0));
  const double uc = us[v];
  const double Au = wr * (uc - us[v + 1]) + wl * (uc - us[v - 1]) + wu * (uc - us[v + N]) + wd * (uc - us[v - N]);
  double load;
  if (c) {
    load = c[lo * N * N + v];
  } else {
    const int NH = (N + 1) / 2;
    const double* f = fH + lo * NH * NH;
    const int a = i >> 1, b = j >> 1;
    if (!(i & 1) && !(j & 1)) load = f[b * NH + a];
    else if (!(j & 1)) load = 0.5 * (f[b * NH + a] + f[b * NH + a + 1]);             // horizontal edge
    else if (!(i & 1)) load = 0.5 * (f[b * NH + a] + f[(b + 1) * NH + a]);            // vertical edge
    else load = 0.5 * (f[b * NH + a] + f[(b + 1) * NH + a + 1]);                     // "/" diagonal
    load *= D.h2;
  }
  rs[v] = load - Au;
}

// Right-hand-side sweep of one node for the group's loads: one warp per (node,
// sample).  z_k over the front rows [gamma, B]: r_k at the node's own gamma rows
// plus the sons' condensed right-hand sides (Eq. block_equation4 positions);
// forward substitution with L_gg leaves y_g (to d_k at the gamma vertices) and
// z_B - L_Bg y_g (to the node's slot for its father).
template <typename T, int R>
__global__ void __launch_bounds__(32 * kDataWarps) k_data_forward(const DataArgs D, const int32_t* __restrict__ list,
                                                                int wstride) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * (blockDim.x >> 5) + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw) + (size_t)warp * wstride * R;   // z_k at z + k * wstride
  if (s >= D.batch) return;
  const NodeDev nd = D.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = D.maps + nd.map_off;
  const int64_t NN = (int64_t)D.N * D.N;
  const double* rs = D.r + (int64_t)s * NN;
  const int64_t rk = (int64_t)D.batch * NN;   // between loads
  if (nd.leaf) {
    for (int r = lane; r < nf - 1; r += 32)
#pragma unroll
      for (int k = 0; k < R; ++k) z[k * wstride + r] = (r < m && k < D.nk) ? (T)rs[k * rk + vid[r]] : (T)0;
  } else {
    const NodeDev c0 = D.nodes[nd.child0], c1 = D.nodes[nd.child1];
    const int32_t* pos0 = vid + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    for (int r = lane; r < nf - 1; r += 32) {
      const int q0 = pos0[r], q1 = pos1[r];
#pragma unroll
      for (int k = 0; k < R; ++k) {
        double v = 0.0;
        if (k < D.nk) {
          if (r < m) v = rs[k * rk + vid[r]];
          if (q0 >= 0) v += son_cond(D.A, c0, s, k, q0);
          if (q1 >= 0) v += son_cond(D.A, c1, s, k, q1);
        }
        z[k * wstride + r] = (T)v;
      }
    }
  }
  __syncwarp();
  const T* F = dat_F<T>(D.A, nd, s);
  for (int c = 0; c < m; ++c) {
    const T* col = F + (int64_t)c * nf;
    const T inv = (T)1 / col[c];
    T y[R];
#pragma unroll
    for (int k = 0; k < R; ++k) y[k] = z[k * wstride + c] * inv;
    for (int i = c + 1 + lane; i < nf - 1; i += 32) {
      const T f = col[i];
#pragma unroll
      for (int k = 0; k < R; ++k) z[k * wstride + i] -= f * y[k];
    }
    __syncwarp();
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < R; ++k) z[k * wstride + c] = y[k];
    __syncwarp();
  }
  double* ds = D.d + (int64_t)s * NN;
  for (int c = lane; c < m; c += 32)
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (k < D.nk) ds[k * rk + vid[c]] = (double)z[k * wstride + c];
  if (b > 0) {
    T* slot = dat_slot<T>(D.A, nd, s);
    for (int r = lane; r < b; r += 32)
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (k < D.nk) slot[k * b + r] = z[k * wstride + m + r];
  }
}

// Descent of one node for the group's loads (one warp per (node, sample)):
// t = y_g - L_Bg^T d_B, then L_gg^T d_g = t by back substitution; y_g comes from
// d at the gamma vertices, where d_g replaces it.
template <typename T, int R>
__global__ void __launch_bounds__(32 * kDataWarps) k_data_descent(const DataArgs D, const int32_t* __restrict__ list,
                                                                int wstride) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * (blockDim.x >> 5) + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw) + (size_t)warp * wstride * R;   // [gamma, B] of load k at w + k * wstride
  if (s >= D.batch) return;
  const NodeDev nd = D.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = D.maps + nd.map_off;
  const int64_t NN = (int64_t)D.N * D.N, rk = (int64_t)D.batch * NN;
  double* ds = D.d + (int64_t)s * NN;
  for (int r = lane; r < nf - 1; r += 32)
#pragma unroll
    for (int k = 0; k < R; ++k) w[k * wstride + r] = (k < D.nk) ? (T)ds[k * rk + vid[r]] : (T)0;
  __syncwarp();
  const T* F = dat_F<T>(D.A, nd, s);
  for (int c = m - 1; c >= 0; --c) {
    const T* col = F + (int64_t)c * nf;
    T acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = (T)0;
    for (int r = c + 1 + lane; r < nf - 1; r += 32) {
      const T f = col[r];
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] += f * w[k * wstride + r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] += __shfl_xor_sync(kAll, acc[k], o);
    const T inv = (T)1 / col[c];
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < R; ++k) w[k * wstride + c] = (w[k * wstride + c] - acc[k]) * inv;
    __syncwarp();
  }
  for (int c = lane; c < m; c += 32)
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (k < D.nk) ds[k * rk + vid[c]] = (double)w[k * wstride + c];
}

// The same two sweeps for nodes with long interfaces (m >= kDataCtaMinM): one CTA
// of 256 threads per (node, sample), the interface in 32-column blocks.  Forward:
// warp 0 solves a block's diagonal triangle for the group's loads (shuffles), then
// every thread folds the block into its rows below, reading each factor entry once
// for all loads.  Descent: t = y_g - L_Bg^T d_B with four columns per warp and pass
// (lanes down the boundary rows), then back substitution block by block (warp 0 on
// the diagonal triangle, every warp folding the block into the columns before it).
constexpr int kDataCtaMinM = 16;

template <typename T, int R>
__global__ void __launch_bounds__(256) k_data_forward_cta(const DataArgs D, const int32_t* __restrict__ list,
                                                          int wstride) {
  const int node = list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = D.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = D.maps + nd.map_off;
  const int64_t NN = (int64_t)D.N * D.N, rk = (int64_t)D.batch * NN;
  const double* rs = D.r + (int64_t)s * NN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw);   // load k at z + k * wstride
  T* Ld = z + R * wstride;                 // [32][33] diagonal block of L_gg
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (nd.leaf) {
    for (int r = threadIdx.x; r < nf - 1; r += blockDim.x)
#pragma unroll
      for (int k = 0; k < R; ++k) z[k * wstride + r] = (r < m && k < D.nk) ? (T)rs[k * rk + vid[r]] : (T)0;
  } else {
    const NodeDev c0 = D.nodes[nd.child0], c1 = D.nodes[nd.child1];
    const int32_t* pos0 = vid + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    for (int r = threadIdx.x; r < nf - 1; r += blockDim.x) {
      const int q0 = pos0[r], q1 = pos1[r];
#pragma unroll
      for (int k = 0; k < R; ++k) {
        double v = 0.0;
        if (k < D.nk) {
          if (r < m) v = rs[k * rk + vid[r]];
          if (q0 >= 0) v += son_cond(D.A, c0, s, k, q0);
          if (q1 >= 0) v += son_cond(D.A, c1, s, k, q1);
        }
        z[k * wstride + r] = (T)v;
      }
    }
  }
  const T* F = dat_F<T>(D.A, nd, s);
  for (int cb = 0; cb < m; cb += 32) {
    const int jb = min(32, m - cb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * jb; idx += blockDim.x) {
      const int c = idx >> 5, l = idx & 31;
      Ld[c * 33 + l] = (l < jb) ? F[(int64_t)(cb + c) * nf + cb + l] : (T)0;
    }
    __syncthreads();
    if (warp == 0) {
      T x[R];
#pragma unroll
      for (int k = 0; k < R; ++k) x[k] = (lane < jb) ? z[k * wstride + cb + lane] : (T)0;
      for (int c = 0; c < jb; ++c) {
        const T dc = Ld[c * 33 + c], lc = Ld[c * 33 + lane];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const T yc = __shfl_sync(kAll, x[k], c) / dc;
          if (lane == c) x[k] = yc;
          if (lane > c && lane < jb) x[k] -= lc * yc;
        }
      }
      if (lane < jb)
#pragma unroll
        for (int k = 0; k < R; ++k) z[k * wstride + cb + lane] = x[k];
    }
    __syncthreads();
    for (int i = cb + jb + threadIdx.x; i < nf - 1; i += blockDim.x) {
      T acc[R];
#pragma unroll
      for (int k = 0; k < R; ++k) acc[k] = (T)0;
      for (int c = 0; c < jb; ++c) {
        const T f = F[(int64_t)(cb + c) * nf + i];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] += f * z[k * wstride + cb + c];
      }
#pragma unroll
      for (int k = 0; k < R; ++k) z[k * wstride + i] -= acc[k];
    }
  }
  __syncthreads();
  double* ds = D.d + (int64_t)s * NN;
  for (int c = threadIdx.x; c < m; c += blockDim.x)
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (k < D.nk) ds[k * rk + vid[c]] = (double)z[k * wstride + c];
  if (b > 0) {
    T* slot = dat_slot<T>(D.A, nd, s);
    for (int r = threadIdx.x; r < b; r += blockDim.x)
#pragma unroll
      for (int k = 0; k < R; ++k)
        if (k < D.nk) slot[k * b + r] = z[k * wstride + m + r];
  }
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_data_descent_cta(const DataArgs D, const int32_t* __restrict__ list,
                                                          int wstride) {
  const int node = list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = D.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = D.maps + nd.map_off;
  const int64_t NN = (int64_t)D.N * D.N, rk = (int64_t)D.batch * NN;
  double* ds = D.d + (int64_t)s * NN;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);   // [gamma (t, then d_g), B (d_B)] of load k at w + k * wstride
  T* Ld = w + R * wstride;                 // [32][33]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int r = threadIdx.x; r < nf - 1; r += blockDim.x)
#pragma unroll
    for (int k = 0; k < R; ++k) w[k * wstride + r] = (k < D.nk) ? (T)ds[k * rk + vid[r]] : (T)0;
  __syncthreads();
  const T* F = dat_F<T>(D.A, nd, s);
  // t_c = y_c - sum_i F[m + i, c] d_B,i: four columns per warp and pass, lanes down the rows
  for (int c0 = 4 * warp; c0 < m; c0 += 4 * nwarp) {
    T acc[4][R];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int k = 0; k < R; ++k) acc[q][k] = (T)0;
    for (int i = lane; i < b; i += 32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T f = (c0 + q < m) ? F[(int64_t)(c0 + q) * nf + m + i] : (T)0;
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] += f * w[k * wstride + m + i];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] += __shfl_xor_sync(kAll, acc[q][k], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c0 + q < m)
#pragma unroll
          for (int k = 0; k < R; ++k) w[k * wstride + c0 + q] -= acc[q][k];
  }
  // back substitution L_gg^T d_g = t, last block first
  for (int cb = ((m - 1) / 32) * 32; cb >= 0; cb -= 32) {
    const int jb = min(32, m - cb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * jb; idx += blockDim.x) {
      const int c = idx >> 5, l = idx & 31;
      Ld[c * 33 + l] = (l < jb) ? F[(int64_t)(cb + c) * nf + cb + l] : (T)0;
    }
    __syncthreads();
    if (warp == 0) {
      T x[R];
#pragma unroll
      for (int k = 0; k < R; ++k) x[k] = (lane < jb) ? w[k * wstride + cb + lane] : (T)0;
      for (int r = jb - 1; r >= 0; --r) {
        const T dr = Ld[r * 33 + r], lr = Ld[lane * 33 + r];
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const T ur = __shfl_sync(kAll, x[k], r) / dr;
          if (lane == r) x[k] = ur;
          if (lane < r) x[k] -= lr * ur;
        }
      }
      if (lane < jb)
#pragma unroll
        for (int k = 0; k < R; ++k) w[k * wstride + cb + lane] = x[k];
    }
    __syncthreads();
    // fold the block into the columns before it: t_c -= sum_l F[cb + l, c] d_{cb + l}
    for (int c0 = 4 * warp; c0 < cb; c0 += 4 * nwarp) {
      T acc[4][R];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) {
          acc[q][k] = (c0 + q < cb && lane < jb) ? F[(int64_t)(c0 + q) * nf + cb + lane] * w[k * wstride + cb + lane]
                                                 : (T)0;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int k = 0; k < R; ++k) acc[q][k] += __shfl_xor_sync(kAll, acc[q][k], o);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c0 + q < cb)
#pragma unroll
            for (int k = 0; k < R; ++k) w[k * wstride + c0 + q] -= acc[q][k];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x)
#pragma unroll
    for (int k = 0; k < R; ++k)
      if (k < D.nk) ds[k * rk + vid[c]] = (double)w[k * wstride + c];
}

// Condensed leaves (G = K_gg^-1 and one coupling weight per boundary row): one
// half-warp per (leaf, sample), the group's loads in turn.  Forward: y = G r_g
// (to d at the interior vertices), condensed -w_i y[c_i]; descent:
// d_g = y - sum_i (w_i d_B,i) G[:, c_i].
template <typename T>
__global__ void __launch_bounds__(256) k_data_leaf(const DataArgs D, const int32_t* __restrict__ list, int descent) {
  const int node = list[blockIdx.x];
  const int hw = threadIdx.x >> 4, r = threadIdx.x & 15;
  const int s = blockIdx.y * 16 + hw;
  const bool active = s < D.batch;   // both half-warps stay for the shuffles
  const int ss = active ? s : 0;
  const NodeDev nd = D.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = D.maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const T* G = dat_F<T>(D.A, nd, ss);
  const int g_elems = m * (m + 1) / 2;
  const int64_t NN = (int64_t)D.N * D.N, rk = (int64_t)D.batch * NN;
  for (int k = 0; k < D.nk; ++k) {
    double* ds = D.d + k * rk + (int64_t)ss * NN;
    if (!descent) {
      const T z = (r < m) ? (T)D.r[k * rk + (int64_t)ss * NN + vid[r]] : (T)0;
      T v = (T)0;
#pragma unroll
      for (int j = 0; j < kLeafInvMax; ++j) {
        const T zj = __shfl_sync(kAll, z, j, 16);
        if (r < m && j < m) v += G[r >= j ? pk(r, j, m) : pk(j, r, m)] * zj;
      }
      if (active && r < m) ds[vid[r]] = (double)v;
      T* slot = dat_slot<T>(D.A, nd, ss);
      for (int i0 = 0; i0 < b; i0 += 16) {
        const int i = i0 + r;
        const int ci = (i < b) ? cpl[i] : -1;
        const T vc = __shfl_sync(kAll, v, ci >= 0 ? ci : 0, 16);
        if (active && i < b) slot[k * b + i] = (ci >= 0) ? -G[g_elems + i] * vc : (T)0;
      }
    } else {
      T acc = (r < m) ? (T)ds[vid[r]] : (T)0;
      for (int i = 0; i < b; ++i) {
        const int ci = cpl[i];
        if (ci >= 0 && r < m) acc -= G[g_elems + i] * (T)ds[vid[m + i]] * G[r >= ci ? pk(r, ci, m) : pk(ci, r, m)];
      }
      __syncwarp();
      if (active && r < m) ds[vid[r]] = (double)acc;
    }
  }
}

// u_k += d_k at the interior vertices; with `track`, per sample the largest |d| and
// |u| of the group (as ordered bits of non-negative doubles) for the refinement's test.
__global__ void k_data_update(const DataArgs D, int k0, int track) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y, k = blockIdx.z;
  const int N = D.N;
  double dm = 0.0, um = 0.0;
  if (v < N * N) {
    const int i = v % N, j = v / N;
    if (i >= 1 && j >= 1 && i <= N - 2 && j <= N - 2) {
      const int64_t o = ((int64_t)s * D.n_loads + k0 + k) * N * N + v;
      const double dd = D.d[((int64_t)k * D.batch + s) * N * N + v];
      const double un = D.u[o] + dd;
      D.u[o] = un;
      dm = fabs(dd);
      um = fabs(un);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dm = fmax(dm, __shfl_xor_sync(kAll, dm, o));
    um = fmax(um, __shfl_xor_sync(kAll, um, o));
  }
  if (track && (threadIdx.x & 31) == 0 && (dm > 0.0 || um > 0.0)) {
    atomicMax(reinterpret_cast<unsigned long long*>(D.conv + 4 * s), __double_as_longlong(dm));
    atomicMax(reinterpret_cast<unsigned long long*>(D.conv + 4 * s + 1), __double_as_longlong(um));
  }
}

// After each refinement step of a group: the step's largest correction d_K against
// the previous one; after the last, the remaining error d_K min(1, d_K / d_{K-1})
// against tol * max |u| (HDD_ENOCONV otherwise).  conv[4 s + 0..3]: this step's
// max |d|, max |u|, the previous step's max |d|, and a flag that a previous step exists.
__global__ void k_data_conv(const DataArgs D, double tol, int last) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= D.batch) return;
  double* cv = D.conv + 4 * s;
  const double d = cv[0], um = cv[1];
  if (last) {
    const double est = (cv[3] != 0.0 && cv[2] > 0.0) ? d * fmin(1.0, d / cv[2]) : d;
    if (!(est <= tol * um) && D.status) atomicCAS(D.status + s, 0, -HDD_ENOCONV);
    cv[2] = cv[3] = 0.0;
  } else {
    cv[2] = d;
    cv[3] = 1.0;
  }
  cv[0] = cv[1] = 0.0;
}


cudaError_t launch_data_init(const DataArgs& D, const double* g, int k0, cudaStream_t st) {
  const int NN = D.N * D.N;
  k_data_init<<<dim3((NN + 255) / 256, D.batch, D.nk), 256, 0, st>>>(D, g, k0);
  return cudaGetLastError();
}
cudaError_t launch_data_residual(const DataArgs& D, const double* kappa, int64_t kap_stride, const double* c,
                                 const double* fH, int k0, cudaStream_t st) {
  const int NN = D.N * D.N;
  k_data_residual<<<dim3((NN + 127) / 128, D.batch, D.nk), 128, 0, st>>>(D, kappa, kap_stride, c, fH, k0);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_data_sweep(const DataArgs& D, const int32_t* list, int nlist, int max_nf, int max_m, bool descent,
                              cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  const int ws = (max_nf + 3) & ~3;
  if (max_m >= kDataCtaMinM) {   // long interfaces: one CTA per (node, sample)
    const size_t smem = ((size_t)kData * ws + 32 * 33) * sizeof(T);
    if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    const dim3 grid(nlist, D.batch);
    if (descent) k_data_descent_cta<T, kData><<<grid, 256, smem, st>>>(D, list, ws);
    else k_data_forward_cta<T, kData><<<grid, 256, smem, st>>>(D, list, ws);
    return cudaGetLastError();
  }
  const size_t per_warp = (size_t)kData * ws * sizeof(T);
  int wpb = kDataWarps;
  while (wpb > 1 && (size_t)wpb * per_warp > 227 * 1024) --wpb;
  if (per_warp > 227 * 1024) return cudaErrorInvalidConfiguration;
  const dim3 grid(nlist, (D.batch + wpb - 1) / wpb);
  if (descent) k_data_descent<T, kData><<<grid, 32 * wpb, wpb * per_warp, st>>>(D, list, ws);
  else k_data_forward<T, kData><<<grid, 32 * wpb, wpb * per_warp, st>>>(D, list, ws);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_data_leaf(const DataArgs& D, const int32_t* list, int nlist, bool descent, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_data_leaf<T><<<dim3(nlist, (D.batch + 15) / 16), 256, 0, st>>>(D, list, descent ? 1 : 0);
  return cudaGetLastError();
}
cudaError_t launch_data_update(const DataArgs& D, int k0, double tol, bool last, bool test, cudaStream_t st) {
  const int NN = D.N * D.N;
  k_data_update<<<dim3((NN + 255) / 256, D.batch, D.nk), 256, 0, st>>>(D, k0, test ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && test) {
    k_data_conv<<<(D.batch + 127) / 128, 128, 0, st>>>(D, tol, last ? 1 : 0);
    e = cudaGetLastError();
  }
  return e;
}
template cudaError_t launch_data_sweep<double>(const DataArgs&, const int32_t*, int, int, int, bool, cudaStream_t);
template cudaError_t launch_data_sweep<float>(const DataArgs&, const int32_t*, int, int, int, bool, cudaStream_t);
template cudaError_t launch_data_leaf<double>(const DataArgs&, const int32_t*, int, bool, cudaStream_t);
template cudaError_t launch_data_leaf<float>(const DataArgs&, const int32_t*, int, bool, cudaStream_t);

cudaError_t configure_data_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_data_forward<double, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_forward<float, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_descent<double, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_descent<float, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_forward_cta<double, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_forward_cta<float, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_descent_cta<double, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_data_descent_cta<float, kData>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
