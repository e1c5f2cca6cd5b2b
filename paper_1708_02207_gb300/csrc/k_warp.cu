// Right-hand-side and descent sweeps with one warp per (node, sample).  A CTA
// of 8 warps serves 8 samples of the same node, which share the node's index
// maps.
#include "launch.h"

namespace hdd {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> __device__ __forceinline__ T* warp_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* warp_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* warp_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* warp_S(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* warp_S<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* warp_S<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

// A warp copies n consecutive values from global to shared memory with eight
// loads in flight per lane (all issued before the stores).
template <typename T>
__device__ __forceinline__ void warp_stage(T* dst, const T* __restrict__ src, int n, int lane) {
  constexpr int U = 8;
  int i = lane;
  for (; i + 32 * (U - 1) < n; i += 32 * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = src[i + 32 * u];
#pragma unroll
    for (int u = 0; u < U; ++u) dst[i + 32 * u] = v[u];
  }
  for (; i < n; i += 32) dst[i] = src[i];
}

// Warps per CTA of the sweeps: 8, or fewer when a warp's vector of nf entries
// would not fit the shared memory of 8 warps.
static int sweep_warps(size_t bytes_per_warp) {
  const size_t lim = 227 * 1024;
  int w = 8;
  while (w > 1 && (size_t)w * bytes_per_warp > lim) --w;
  return w;
}

// ---------------------------------------------------------------------------
// Right-hand-side sweep at one node (leaves to root), one warp per sample:
// z = sons' condensed right-hand sides + r at gamma; y = L_gg^-1 z_g column by
// column, folding every column into the rows below it, which leaves z_B - L_Bg y_g.
// The node's factor block is first staged in shared memory with coalesced loads
// (all in flight at once), so the sequential solve runs on shared memory.
// Outputs: y_g into the y arena, the condensed right-hand side (b entries)
// contiguously at the start of the node's (now unused) Schur block.
template <typename T>
__device__ __forceinline__ T son_cond(const Arenas& A, const NodeDev& ch, int s, int p) {
  const int64_t idx = (int64_t)p + ch.s_off;
  return ch.fp64 ? (T)A.s64[(int64_t)s * A.s64_stride + idx] : (T)A.s32[(int64_t)s * A.s32_stride + idx];
}

template <typename T>
__global__ void __launch_bounds__(256) k_forward_warp(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, int wstride,
                                                      int stage, Arenas A, Rhs rhs) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * (blockDim.x >> 5) + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* z = reinterpret_cast<T*>(smem_raw) + warp * wstride;
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const T* Fg = warp_F<T>(A, nd, s);
  const T* F = Fg;
  if (stage) {
    T* Fs = z + ((nf + 3) & ~3);
    warp_stage(Fs, Fg, nf * m, lane);
    F = Fs;
  }
  if (nd.leaf) {
    for (int r = lane; r < nf - 1; r += 32) z[r] = (r < m) ? (T)rhs(s, vid[r]) : (T)0;
  } else {
    const NodeDev c0 = nodes[nd.child0], c1 = nodes[nd.child1];
    const int32_t* pos0 = vid + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    for (int r = lane; r < nf - 1; r += 32) {
      T val = (r < m) ? (T)rhs(s, vid[r]) : (T)0;
      const int q0 = pos0[r], q1 = pos1[r];
      if (q0 >= 0) val += son_cond<T>(A, c0, s, q0);
      if (q1 >= 0) val += son_cond<T>(A, c1, s, q1);
      z[r] = val;
    }
  }
  __syncwarp();
  for (int c = 0; c < m; ++c) {
    const T* col = F + (int64_t)c * nf;
    const T yc = z[c] / col[c];
    for (int i = c + 1 + lane; i < nf - 1; i += 32) z[i] -= col[i] * yc;
    __syncwarp();
    if (lane == 0) z[c] = yc;
    __syncwarp();
  }
  T* Y = node_Y<T>(A, nd, s);
  for (int c = lane; c < m; c += 32) Y[c] = z[c];
  if (b > 0) {
    T* S = warp_S<T>(A, nd, s);
    for (int r = lane; r < b; r += 32) S[r] = z[m + r];
  }
}

// Bytes of shared memory per warp of a sweep: the vector, plus the staged
// factor block when it fits in 64 KiB.
template <typename T>
static int sweep_stride(int max_nf, int max_m, int* stage) {
  const size_t vec = (size_t)((max_nf + 3) & ~3);
  const size_t fac = (size_t)max_nf * max_m;
  const size_t yg = (size_t)((max_m + 3) & ~3);   // y_g (descent)
  *stage = (vec + fac + yg) * sizeof(T) <= 64 * 1024;
  return (int)(*stage ? vec + fac + yg : vec + yg);
}

template <typename T>
cudaError_t launch_forward_warp(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, int max_nf, int max_m, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  int stage = 0;
  const int ws = sweep_stride<T>(max_nf, max_m, &stage);
  const int wpb = sweep_warps((size_t)ws * sizeof(T));
  k_forward_warp<T><<<dim3(nlist, (batch + wpb - 1) / wpb), 32 * wpb, (size_t)wpb * ws * sizeof(T), st>>>(
      nodes, maps, list, batch, ws, stage, A, rhs);
  return cudaGetLastError();
}
template cudaError_t launch_forward_warp<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, const Rhs&, int, int, cudaStream_t);
template cudaError_t launch_forward_warp<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, const Rhs&, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Descent at one node (Root to Leaves), one warp per sample: with w = [u_g; u_B]
// (u_B gathered from the vertex vector), for c = m-1 .. 0
//   u_c = (y_c - sum_{r > c} F[r, c] w_r) / F[c, c],
// i.e. L_gg^T u_g = y_g - L_Bg^T u_B; the factor block is staged first.
template <typename T>
__global__ void __launch_bounds__(256) k_descent_warp(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, int wstride,
                                                      int stage, Arenas A, double* __restrict__ u, int64_t u_stride) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * (blockDim.x >> 5) + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* wv = reinterpret_cast<T*>(smem_raw) + warp * wstride;
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const T* Fg = warp_F<T>(A, nd, s);
  const T* F = Fg;
  if (stage) {
    T* Fs = wv + ((nf + 3) & ~3);
    warp_stage(Fs, Fg, nf * m, lane);
    F = Fs;
  }
  const T* Y = node_Y<T>(A, nd, s);
  double* us = u + (int64_t)s * u_stride;
  for (int i0 = 0; i0 < b; i0 += 128) {   // u_B: four gathers per lane in flight
    int v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = (i0 + 32 * q + lane < b) ? vid[m + i0 + 32 * q + lane] : -1;
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = v[q] >= 0 ? us[v[q]] : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (v[q] >= 0) wv[m + i0 + 32 * q + lane] = (T)x[q];
  }
  T* ys = wv + ((nf + 3) & ~3) + (stage ? nf * m : 0);   // y_g, staged with the rest
  for (int c = lane; c < m; c += 32) ys[c] = Y[c];
  __syncwarp();
  for (int c = m - 1; c >= 0; --c) {
    const T* col = F + (int64_t)c * nf;
    T acc = (T)0;
    for (int r = c + 1 + lane; r < nf - 1; r += 32) acc += col[r] * wv[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    const T uc = (ys[c] - acc) / col[c];
    if (lane == 0) wv[c] = uc;
    __syncwarp();
  }
  for (int c = lane; c < m; c += 32) us[vid[c]] = (double)wv[c];
}

template <typename T>
cudaError_t launch_descent_warp(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, int max_nf, int max_m,
                                cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  int stage = 0;
  const int ws = sweep_stride<T>(max_nf, max_m, &stage);
  const int wpb = sweep_warps((size_t)ws * sizeof(T));
  k_descent_warp<T><<<dim3(nlist, (batch + wpb - 1) / wpb), 32 * wpb, (size_t)wpb * ws * sizeof(T), st>>>(
      nodes, maps, list, batch, ws, stage, A, u, u_stride);
  return cudaGetLastError();
}
template cudaError_t launch_descent_warp<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, double*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_descent_warp<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, double*, int64_t, int, int, cudaStream_t);


// ---------------------------------------------------------------------------
// Sweeps over fronts of at most 32 rows with the node's factor rows in registers
// (lane r holds row r of F, m <= 31 columns), one warp per (node, sample):
// forward substitution and the descent's dot products by shuffles, without
// shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_forward_tiny(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, Arenas A,
                                                      Rhs rhs) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * 8 + warp;
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const T* F = warp_F<T>(A, nd, s);
  T row[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) row[c] = (c < m && lane < nf - 1) ? F[c * nf + lane] : (T)0;
  T z = (T)0;
  if (lane < nf - 1) {
    if (lane < m) z = (T)rhs(s, vid[lane]);
    if (!nd.leaf) {
      const int32_t* pos0 = vid + (nf - 1);
      const int32_t* pos1 = pos0 + nf;
      const int q0 = pos0[lane], q1 = pos1[lane];
      if (q0 >= 0) z += son_cond<T>(A, nodes[nd.child0], s, q0);
      if (q1 >= 0) z += son_cond<T>(A, nodes[nd.child1], s, q1);
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    if (c >= m) break;    // warp-uniform
    const T d = __shfl_sync(kFull, row[c], c);
    const T yc = __shfl_sync(kFull, z, c) / d;
    if (lane == c) z = yc;
    if (lane > c) z -= row[c] * yc;
  }
  if (lane < m) node_Y<T>(A, nd, s)[lane] = z;
  if (lane >= m && lane < nf - 1) warp_S<T>(A, nd, s)[lane - m] = z;
  (void)b;
}

template <typename T>
__global__ void __launch_bounds__(256) k_descent_tiny(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, Arenas A,
                                                      double* __restrict__ u, int64_t u_stride) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * 8 + warp;
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const T* F = warp_F<T>(A, nd, s);
  double* us = u + (int64_t)s * u_stride;
  T row[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) row[c] = (c < m && lane < nf - 1) ? F[c * nf + lane] : (T)0;
  T wv = (lane >= m && lane < nf - 1) ? (T)us[vid[lane]] : (T)0;   // u_B; u_g filled below
  const T yl = (lane < m) ? node_Y<T>(A, nd, s)[lane] : (T)0;
#pragma unroll
  for (int c = 31; c >= 0; --c) {
    if (c >= m) continue;    // warp-uniform
    T t = (lane > c) ? row[c] * wv : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    const T d = __shfl_sync(kFull, row[c], c);
    const T uc = (__shfl_sync(kFull, yl, c) - t) / d;
    if (lane == c) wv = uc;
  }
  if (lane < m) us[vid[lane]] = (double)wv;
}

template <typename T>
cudaError_t launch_forward_tiny(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_forward_tiny<T><<<dim3(nlist, (batch + 7) / 8), 256, 0, st>>>(nodes, maps, list, batch, A, rhs);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_descent_tiny(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_descent_tiny<T><<<dim3(nlist, (batch + 7) / 8), 256, 0, st>>>(nodes, maps, list, batch, A, u, u_stride);
  return cudaGetLastError();
}
template cudaError_t launch_forward_tiny<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, const Rhs&, cudaStream_t);
template cudaError_t launch_forward_tiny<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, const Rhs&, cudaStream_t);
template cudaError_t launch_descent_tiny<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, double*, int64_t, cudaStream_t);
template cudaError_t launch_descent_tiny<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, double*, int64_t, cudaStream_t);

// ---------------------------------------------------------------------------
// Right-hand-side sweep over fronts of 16..32 eliminated vertices and at most 256 rows
// (the middle levels of the tree), one warp per (node, sample), eight samples of a node
// per CTA.  Lane l owns rows l + 32 j of the front (j < kMidJ) in registers: z = load at
// gamma + sons' condensed loads; for each column c, y_c = z_c / F[c, c] and the column
// folded into the rows below it, the next column's entries loaded while the current
// one is applied, so no front is staged whole.
constexpr int kMidJ = 8;   // rows per lane: fronts of up to 256 rows

template <typename T>
__global__ void __launch_bounds__(256) k_forward_mid(const NodeDev* __restrict__ nodes,
                                                     const int32_t* __restrict__ maps,
                                                     const int32_t* __restrict__ list, int batch, Arenas A,
                                                     Rhs rhs) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * 8 + warp;
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, nr = nd.nf - 1, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const T* F = warp_F<T>(A, nd, s);
  T z[kMidJ];
  {
    const NodeDev c0 = nd.leaf ? nd : nodes[nd.child0], c1 = nd.leaf ? nd : nodes[nd.child1];
    const int32_t* pos0 = vid + nr;
    const int32_t* pos1 = pos0 + nf;
#pragma unroll
    for (int j = 0; j < kMidJ; ++j) {
      const int r = lane + 32 * j;
      T v = (T)0;
      if (r < nr) {
        if (r < m) v = (T)rhs(s, vid[r]);
        if (!nd.leaf) {
          const int q0 = pos0[r], q1 = pos1[r];
          if (q0 >= 0) v += son_cond<T>(A, c0, s, q0);
          if (q1 >= 0) v += son_cond<T>(A, c1, s, q1);
        }
      }
      z[j] = v;
    }
  }
  T f[kMidJ];   // column c of F at this lane's rows
#pragma unroll
  for (int j = 0; j < kMidJ; ++j) {
    const int r = lane + 32 * j;
    f[j] = r < nr ? F[r] : (T)0;
  }
  for (int c = 0; c < m; ++c) {
    T fn[kMidJ];   // the next column, in flight while this one is applied
#pragma unroll
    for (int j = 0; j < kMidJ; ++j) {
      const int r = lane + 32 * j;
      fn[j] = (c + 1 < m && r < nr) ? F[(int64_t)(c + 1) * nf + r] : (T)0;
    }
    if (lane == c) z[0] = z[0] / f[0];   // F[c, c] at lane c
    const T yc = __shfl_sync(kFull, z[0], c);
#pragma unroll
    for (int j = 0; j < kMidJ; ++j) {
      const int r = lane + 32 * j;
      if (r > c && r < nr) z[j] -= f[j] * yc;
    }
#pragma unroll
    for (int j = 0; j < kMidJ; ++j) f[j] = fn[j];
  }
  if (lane < m) node_Y<T>(A, nd, s)[lane] = z[0];
  if (nd.b > 0) {
    T* S = warp_S<T>(A, nd, s);
#pragma unroll
    for (int j = 0; j < kMidJ; ++j) {
      const int r = lane + 32 * j;
      if (r >= m && r < nr) S[r - m] = z[j];
    }
  }
}

template <typename T>
cudaError_t launch_forward_mid(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                               const Arenas& A, const Rhs& rhs, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_forward_mid<T><<<dim3(nlist, (batch + 7) / 8), 256, 0, st>>>(nodes, maps, list, batch, A, rhs);
  return cudaGetLastError();
}
template cudaError_t launch_forward_mid<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, const Rhs&, cudaStream_t);
template cudaError_t launch_forward_mid<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                               const Arenas&, const Rhs&, cudaStream_t);

}  // namespace hdd

namespace hdd {
cudaError_t configure_warp_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_forward_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_forward_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_descent_warp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_descent_warp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}
}  // namespace hdd
