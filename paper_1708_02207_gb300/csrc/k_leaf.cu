// Condensed leaves.  A leaf with m <= kLeafInvMax interior vertices eliminates
// its interior by the explicit inverse G = K_gg^-1 instead of keeping the
// partial Cholesky factors: on this mesh every boundary vertex i of a leaf
// rectangle couples to at most one interior vertex c_i, with the stiffness
// entry w_i = K_Bg[i, c_i] (Eq. coefA: minus the weight of the shared edge), so
// the Schur maps of the leaf (Sec. 2.4, Eq. SchurC1) reduce to
//   S_ij      = K_BB[i, j] - w_i w_j G[c_i, c_j]            (boundary block)
//   z_B,i     = -w_i (G b_g)[c_i]                           (condensed load)
//   u_g       = G b_g - sum_i w_i u_B,i G[:, c_i]           (descent, "Root to Leaves")
// which is the same elimination in exact arithmetic.  Per sample the factor
// store holds G (packed lower, column-major) followed by w [b]; y_g holds
// G b_g.  One warp per (leaf, sample), eight samples of one leaf per CTA.
#include "launch.h"

namespace hdd {

namespace {

constexpr unsigned kAllLanes = 0xffffffffu;
constexpr int kLd = kLeafInvMax + 1;   // row stride of the per-warp m x m buffers

// packed lower column-major index of (i, j), i >= j, of an m x m matrix
__device__ __forceinline__ int pk(int i, int j, int m) { return j * m - j * (j - 1) / 2 + (i - j); }

template <typename T> __device__ __forceinline__ T* leaf_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* leaf_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* leaf_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* leaf_S(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* leaf_S<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* leaf_S<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

// per-warp shared buffers of the leaf front (elements of T)
constexpr int kWarpElems = 3 * kLeafInvMax * kLd + (kLeafInvMaxB + 1) + kLeafInvMax;

}  // namespace

// Upsweep at condensed leaves: stiffness of the leaf's own triangles (only the
// stencil nonzeros), Cholesky of K_gg in registers (lane r holds row r), W =
// L^-1 by forward substitution (lane c solves L w = e_c), G = W^T W, then G,
// w, y_g = G b_g and the leaf's lower Schur triangle with its condensed load.
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_front(StepArgs a) {
  const int node = a.list[blockIdx.x];
  const NodeDev nd = a.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf, nb = b + 1, N = a.N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * 8 + warp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Kg = reinterpret_cast<T*>(smem_raw) + warp * kWarpElems;   // K_gg, then L (row-major, ld kLd)
  T* Wm = Kg + kLeafInvMax * kLd;                                // W = L^-1 (row-major)
  T* Gs = Wm + kLeafInvMax * kLd;                                // G (full, row-major)
  T* wv = Gs + kLeafInvMax * kLd;                                // w [b]
  T* vs = wv + kLeafInvMaxB + 1;                                 // G b_g [m]
  int* tbl = reinterpret_cast<int*>(reinterpret_cast<T*>(smem_raw) + 8 * kWarpElems);
  const int32_t* vid = a.maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const int tw = nd.x1 - nd.x0 + 1, cells = tw * (nd.y1 - nd.y0 + 1);
  int* loc = tbl + cells;   // local (column, row) of each front row's vertex
  for (int i = threadIdx.x; i < cells; i += blockDim.x) tbl[i] = -1;
  __syncthreads();
  for (int r = threadIdx.x; r < nf - 1; r += blockDim.x) {
    const int v = vid[r];
    const int li = v % N - nd.x0, lj = v / N - nd.y0;
    tbl[lj * tw + li] = r;
    loc[r] = (lj << 16) | li;
  }
  __syncthreads();
  if (s >= a.batch) return;
  const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)s * a.kap_stride;

  // 1. interior rows of the stiffness and the boundary couplings
  for (int i = lane; i < kLeafInvMax * kLd; i += 32) Kg[i] = (T)0;
  for (int i = lane; i < b; i += 32) wv[i] = (T)0;
  __syncwarp();
  T bg = (T)0;   // load of interior vertex `lane` (Eq. coefc)
  if (lane < m) {
    const int li = loc[lane] & 0xffff, lj = loc[lane] >> 16;
    const int vi = nd.x0 + li, vj = nd.y0 + lj;
    const T wl = w_horizontal(kap, N, nd, vi - 1, vj), wr = w_horizontal(kap, N, nd, vi, vj);
    const T wd = w_vertical(kap, N, nd, vi, vj - 1), wu = w_vertical(kap, N, nd, vi, vj);
    Kg[lane * kLd + lane] = wl + wr + wd + wu;
    const int nbr[4] = {li > 0 ? tbl[lj * tw + li - 1] : -1, vi < nd.x1 ? tbl[lj * tw + li + 1] : -1,
                        lj > 0 ? tbl[(lj - 1) * tw + li] : -1, vj < nd.y1 ? tbl[(lj + 1) * tw + li] : -1};
    const T wgt[4] = {wl, wr, wd, wu};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = nbr[q];
      if (c < 0) continue;
      if (c < m) Kg[lane * kLd + c] = -wgt[q];
      else wv[c - m] = -wgt[q];   // the boundary row's only interior neighbour is this vertex
    }
    bg = (T)a.rhs(s, vj * N + vi);
  }
  __syncwarp();

  // 2. Cholesky K_gg = L L^T, lane r holding row r; pivot column by shuffles
  T row[kLeafInvMax];
#pragma unroll
  for (int c = 0; c < kLeafInvMax; ++c) row[c] = (lane < m && c < m) ? Kg[lane * kLd + c] : (T)0;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kLeafInvMax; ++k) {
    if (k < m) {
      T pkk = __shfl_sync(kAllLanes, row[k], k);
      if (!(pkk > (T)0) || !isfinite(pkk)) {   // not SPD: record, continue with a unit pivot
        bad = true;
        pkk = (T)1;
      }
      const T d = sqrt(pkk), inv = (T)1 / d;
      T lk = (lane == k) ? d : row[k] * inv;
      if (lane < k) lk = (T)0;
#pragma unroll
      for (int j = k + 1; j < kLeafInvMax; ++j) {
        const T lj = __shfl_sync(kAllLanes, lk, j);
        if (lane > k) row[j] -= lk * lj;
      }
      row[k] = lk;
    }
  }
  if (bad && lane == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
  if (lane < kLeafInvMax)
#pragma unroll
    for (int c = 0; c < kLeafInvMax; ++c) Kg[lane * kLd + c] = row[c];
  __syncwarp();

  // 3. W = L^-1: lane c solves L w = e_c (rows of L read by all lanes at once)
  T w[kLeafInvMax];
#pragma unroll
  for (int r = 0; r < kLeafInvMax; ++r) {
    T acc = (lane == r) ? (T)1 : (T)0;
#pragma unroll
    for (int l = 0; l < r; ++l) acc -= Kg[r * kLd + l] * w[l];
    w[r] = (r < m) ? acc / Kg[r * kLd + r] : (T)0;
  }
  if (lane < kLeafInvMax)
#pragma unroll
    for (int r = 0; r < kLeafInvMax; ++r) Wm[r * kLd + lane] = w[r];
  __syncwarp();

  // 4. G = W^T W (lane i: row i; W is lower, so w[k] = W[k, i] vanishes for k < i)
  T* F = leaf_F<T>(a.arenas, nd, s);
  if (lane < m) {
#pragma unroll
    for (int j = 0; j < kLeafInvMax; ++j) {
      if (j >= m) break;
      T g = (T)0;
#pragma unroll
      for (int k = 0; k < kLeafInvMax; ++k)
        if (k < m) g += w[k] * Wm[k * kLd + j];
      Gs[lane * kLd + j] = g;
      if (j <= lane) F[pk(lane, j, m)] = g;
    }
  }
  __syncwarp();

  // 5. y_g = G b_g
  T vI = (T)0;
#pragma unroll
  for (int j = 0; j < kLeafInvMax; ++j) {
    const T bj = __shfl_sync(kAllLanes, bg, j);
    if (lane < m && j < m) vI += Gs[lane * kLd + j] * bj;
  }
  if (lane < m) {
    node_Y<T>(a.arenas, nd, s)[lane] = vI;
    vs[lane] = vI;
  }
  const int g_elems = m * (m + 1) / 2;
  for (int i = lane; i < b; i += 32) F[g_elems + i] = wv[i];
  __syncwarp();

  // 6. lower Schur triangle ((b+1) x (b+1), column-major), walked in packed order
  T* S = leaf_S<T>(a.arenas, nd, s);
  const int total = nb * (nb + 1) / 2;
  int c = 0, off = lane;   // entry (c + off, c)
  while (c < nb && off >= nb - c) { off -= nb - c; ++c; }
  for (int t = lane; t < total; t += 32) {
    const int i = c + off, j = c;   // i >= j
    T val = (T)0;
    if (i < b) {
      const int ri = loc[m + i], rj = loc[m + j];
      const int lii = ri & 0xffff, lji = ri >> 16, lij = rj & 0xffff, ljj = rj >> 16;
      const int vi = nd.x0 + lii, vj = nd.y0 + lji;
      if (i == j) {
        val = w_horizontal(kap, N, nd, vi - 1, vj) + w_horizontal(kap, N, nd, vi, vj) +
              w_vertical(kap, N, nd, vi, vj - 1) + w_vertical(kap, N, nd, vi, vj);
      } else if (lji == ljj && (lii - lij == 1 || lij - lii == 1)) {
        val = -w_horizontal(kap, N, nd, nd.x0 + min(lii, lij), vj);
      } else if (lii == lij && (lji - ljj == 1 || ljj - lji == 1)) {
        val = -w_vertical(kap, N, nd, vi, nd.y0 + min(lji, ljj));
      }
      const int ci = cpl[i], cj = cpl[j];
      if (ci >= 0 && cj >= 0) val -= wv[i] * wv[j] * Gs[ci * kLd + cj];
    } else if (j < b) {   // condensed load (bordered row)
      const int cj = cpl[j];
      if (cj >= 0) val = -wv[j] * vs[cj];
    }
    S[j * nb + i] = val;
    off += 32;
    while (c < nb && off >= nb - c) { off -= nb - c; ++c; }
  }
}

// Right-hand-side sweep at condensed leaves: y_g = G r_g, z_B,i = -w_i y_g[c_i]
// (written to the start of the leaf's Schur block, where the father reads it).
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_forward(const NodeDev* __restrict__ nodes,
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
  const int32_t* cpl = vid + (nf - 1);
  const T* F = leaf_F<T>(A, nd, s);
  const T z = (lane < m) ? (T)rhs(s, vid[lane]) : (T)0;
  T v = (T)0;
#pragma unroll
  for (int j = 0; j < kLeafInvMax; ++j) {
    const T zj = __shfl_sync(kAllLanes, z, j);
    if (lane < m && j < m) v += F[lane >= j ? pk(lane, j, m) : pk(j, lane, m)] * zj;
  }
  if (lane < m) node_Y<T>(A, nd, s)[lane] = v;
  T* S = leaf_S<T>(A, nd, s);
  const int g_elems = m * (m + 1) / 2;
  for (int i0 = 0; i0 < b; i0 += 32) {
    const int i = i0 + lane;
    const int ci = (i < b) ? cpl[i] : -1;
    const T vc = __shfl_sync(kAllLanes, v, ci >= 0 ? ci : 0);
    if (i < b) S[i] = (ci >= 0) ? -F[g_elems + i] * vc : (T)0;
  }
}

// Descent at condensed leaves: u_g = y_g - sum_i (w_i u_B,i) G[:, c_i].
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_descent(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, Arenas A,
                                                      double* __restrict__ u, int64_t u_stride) {
  const int node = list[blockIdx.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * 8 + warp;
  __shared__ T tw[8][kLeafInvMaxB + 1];
  __shared__ int cw[8][kLeafInvMaxB + 1];
  if (s >= batch) return;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const T* F = leaf_F<T>(A, nd, s);
  double* us = u + (int64_t)s * u_stride;
  const int g_elems = m * (m + 1) / 2;
  for (int i = lane; i < b; i += 32) {
    cw[warp][i] = cpl[i];
    tw[warp][i] = F[g_elems + i] * (T)us[vid[m + i]];
  }
  __syncwarp();
  if (lane < m) {
    T acc = node_Y<T>(A, nd, s)[lane];
    for (int i = 0; i < b; ++i) {
      const int ci = cw[warp][i];
      if (ci >= 0) acc -= tw[warp][i] * F[lane >= ci ? pk(lane, ci, m) : pk(ci, lane, m)];
    }
    us[vid[lane]] = (double)acc;
  }
}

template <typename T>
cudaError_t launch_leaf_front(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  const size_t smem = (size_t)8 * kWarpElems * sizeof(T) + (size_t)(a.max_rect + a.max_nf) * sizeof(int);
  if (a.prof) a.prof->begin(kProfLeaf, a.fl_chol + a.fl_trsm + a.fl_syrk + a.fl_rhs, st);
  k_leaf_front<T><<<dim3(a.nlist, (a.batch + 7) / 8), 256, smem, st>>>(a);
  if (a.prof) a.prof->end(st);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_leaf_forward(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_leaf_forward<T><<<dim3(nlist, (batch + 7) / 8), 256, 0, st>>>(nodes, maps, list, batch, A, rhs);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_leaf_descent(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_leaf_descent<T><<<dim3(nlist, (batch + 7) / 8), 256, 0, st>>>(nodes, maps, list, batch, A, u, u_stride);
  return cudaGetLastError();
}
template cudaError_t launch_leaf_front<double>(const StepArgs&, cudaStream_t);
template cudaError_t launch_leaf_front<float>(const StepArgs&, cudaStream_t);
template cudaError_t launch_leaf_forward<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, const Rhs&, cudaStream_t);
template cudaError_t launch_leaf_forward<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, const Rhs&, cudaStream_t);
template cudaError_t launch_leaf_descent<double>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                 const Arenas&, double*, int64_t, cudaStream_t);
template cudaError_t launch_leaf_descent<float>(const NodeDev*, const int32_t*, const int32_t*, int, int,
                                                const Arenas&, double*, int64_t, cudaStream_t);

cudaError_t configure_leaf_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_leaf_front<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_leaf_front<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
