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
// G b_g.
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

// per-sample shared buffers of the leaf front (elements of T, then ints)
// The two samples of a warp (its half-warps) sit one stride apart: a stride of 16 words
// modulo the 32 shared-memory banks puts their rows in disjoint banks
constexpr int kSampBase = kLeafInvMax * kLd + 4 * (kLeafInvMaxB + 1) + kLeafInvMax;
template <typename T>
__host__ __device__ constexpr int samp_elems() {
  constexpr int words = sizeof(T) == 4 ? 16 : 8;   // elements that make 16 words
  constexpr int period = sizeof(T) == 4 ? 32 : 16;
  return (kSampBase + period - words - 1) / period * period + words;
}
constexpr int kSampInts = 2 * (kLeafInvMaxB + 1) + 16;
constexpr int kLeafSamples = 16;   // samples per CTA: two per warp, one per half-warp

}  // namespace

// Upsweep at condensed leaves, one half-warp per (leaf, sample): lane r builds
// row r of K_gg (stencil nonzeros of the leaf's own triangles), Gauss-Jordan
// elimination of [K_gg | I] in registers (no pivoting: K_gg is SPD, the pivots
// are those of its Cholesky factorisation) leaves G = K_gg^-1 in the right
// half; then y_g = G b_g and the leaf's lower Schur triangle with its
// condensed load, the boundary block of K read from a sparse row list (a
// boundary vertex has at most two boundary neighbours).
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_front(StepArgs a) {
  const int node = a.list[blockIdx.x];
  bind_plan(a, node);
  const NodeDev nd = a.nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf, nb = b + 1, N = a.N;
  const int hw = threadIdx.x >> 4, r = threadIdx.x & 15;   // half-warp = sample, lane r = row
  const int s = blockIdx.y * kLeafSamples + hw;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kSampElems = samp_elems<T>();
  T* Gs = reinterpret_cast<T*>(smem_raw) + hw * kSampElems;   // K_gg rows, then G (ld kLd)
  T* wv = Gs + kLeafInvMax * kLd;                               // couplings w [b]
  T* dB = wv + kLeafInvMaxB + 1;                                // K_BB diagonal [b]
  T* nw0 = dB + kLeafInvMaxB + 1;                               // K_BB entries to lower boundary rows
  T* nw1 = nw0 + kLeafInvMaxB + 1;
  T* vs = nw1 + kLeafInvMaxB + 1;                               // y_g = G b_g [m]
  int* ints = reinterpret_cast<int*>(reinterpret_cast<T*>(smem_raw) + kLeafSamples * kSampElems);
  int* nj0 = ints + hw * kSampInts;                             // their rows (-1: none)
  int* nj1 = nj0 + kLeafInvMaxB + 1;
  int* tbl = ints + kLeafSamples * kSampInts;
  const int32_t* vid = a.maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const int tw = nd.x1 - nd.x0 + 1, cells = tw * (nd.y1 - nd.y0 + 1);
  int* loc = tbl + cells;   // local (column, row) of each front row's vertex
  for (int i = threadIdx.x; i < cells; i += blockDim.x) tbl[i] = -1;
  __syncthreads();
  for (int q = threadIdx.x; q < nf - 1; q += blockDim.x) {
    const int v = vid[q];
    const int li = v % N - nd.x0, lj = v / N - nd.y0;
    tbl[lj * tw + li] = q;
    loc[q] = (lj << 16) | li;
  }
  __syncthreads();
  const bool active = s < a.batch;   // both half-warps stay for the shuffles
  const int ss = active ? s : 0;
  const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)ss * a.kap_stride;

  // 1. interior rows of the stiffness and the boundary couplings
  for (int i = r; i < kLeafInvMax * kLd; i += 16) Gs[i] = (T)0;
  for (int i = r; i < b; i += 16) wv[i] = (T)0;
  __syncwarp();
  T bg = (T)0;   // load of interior vertex r (Eq. coefc)
  if (r < m) {
    const int li = loc[r] & 0xffff, lj = loc[r] >> 16;
    const int vi = nd.x0 + li, vj = nd.y0 + lj;
    const T wl = w_horizontal(kap, N, nd, vi - 1, vj), wr = w_horizontal(kap, N, nd, vi, vj);
    const T wd = w_vertical(kap, N, nd, vi, vj - 1), wu = w_vertical(kap, N, nd, vi, vj);
    Gs[r * kLd + r] = wl + wr + wd + wu;
    const int nbr[4] = {li > 0 ? tbl[lj * tw + li - 1] : -1, vi < nd.x1 ? tbl[lj * tw + li + 1] : -1,
                        lj > 0 ? tbl[(lj - 1) * tw + li] : -1, vj < nd.y1 ? tbl[(lj + 1) * tw + li] : -1};
    const T wgt[4] = {wl, wr, wd, wu};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = nbr[q];
      if (c < 0) continue;
      if (c < m) Gs[r * kLd + c] = -wgt[q];
      else wv[c - m] = -wgt[q];   // the boundary row's only interior neighbour is this vertex
    }
    bg = (T)a.rhs(ss, vj * N + vi);
  }
  // boundary block of K, sparse: diagonal, and the entries to boundary rows below
  for (int i = r; i < b; i += 16) {
    const int li = loc[m + i] & 0xffff, lj = loc[m + i] >> 16;
    const int vi = nd.x0 + li, vj = nd.y0 + lj;
    const T wl = w_horizontal(kap, N, nd, vi - 1, vj), wr = w_horizontal(kap, N, nd, vi, vj);
    const T wd = w_vertical(kap, N, nd, vi, vj - 1), wu = w_vertical(kap, N, nd, vi, vj);
    dB[i] = wl + wr + wd + wu;
    const int nbr[4] = {li > 0 ? tbl[lj * tw + li - 1] : -1, vi < nd.x1 ? tbl[lj * tw + li + 1] : -1,
                        lj > 0 ? tbl[(lj - 1) * tw + li] : -1, vj < nd.y1 ? tbl[(lj + 1) * tw + li] : -1};
    const T wgt[4] = {wl, wr, wd, wu};
    int j0 = -1, j1 = -1;
    T w0 = (T)0, w1 = (T)0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = nbr[q] - m;   // boundary row of the neighbour
      if (nbr[q] < m || c >= i) continue;
      if (j0 < 0) { j0 = c; w0 = -wgt[q]; }
      else { j1 = c; w1 = -wgt[q]; }
    }
    nj0[i] = j0; nw0[i] = w0;
    nj1[i] = j1; nw1[i] = w1;
  }
  __syncwarp();

  // 2. Gauss-Jordan on [K_gg | I]: lane r holds row r; after pivot k, column k
  // of the left half is e_k and only columns > k of it are still needed, while
  // the right half is nonzero only in columns <= k
  T x[kLeafInvMax], g[kLeafInvMax];
#pragma unroll
  for (int c = 0; c < kLeafInvMax; ++c) {
    x[c] = (r < m && c < m) ? Gs[r * kLd + c] : (T)0;
    g[c] = (T)0;
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < kLeafInvMax; ++k) {
    if (k < m) {   // uniform
      T p = __shfl_sync(kAllLanes, x[k], k, 16);
      if (!(p > (T)0) || !isfinite(p)) {   // not SPD: record, continue with a unit pivot
        bad = true;
        p = (T)1;
      }
      const T inv = (T)1 / p;
      const T f = x[k];
      const bool piv = r == k;
      if (piv) g[k] = (T)1;
#pragma unroll
      for (int c = k + 1; c < kLeafInvMax; ++c) {
        const T pc = __shfl_sync(kAllLanes, x[c], k, 16) * inv;
        x[c] = piv ? pc : x[c] - f * pc;
      }
#pragma unroll
      for (int c = 0; c <= k; ++c) {
        const T pc = __shfl_sync(kAllLanes, g[c], k, 16) * inv;
        g[c] = piv ? pc : g[c] - f * pc;
      }
    }
  }
  if (bad && r == 0 && active) flag_status(a.status, s, -HDD_ENOTSPD, node);

  // 3. G, y_g = G b_g, couplings
  T* F = active ? leaf_F<T>(a.arenas, nd, s) : nullptr;
  __syncwarp();
  T vI = (T)0;
#pragma unroll
  for (int c = 0; c < kLeafInvMax; ++c) {
    const T bc = __shfl_sync(kAllLanes, bg, c, 16);
    if (r < m && c < m) {
      Gs[r * kLd + c] = g[c];
      vI += g[c] * bc;
      if (active && c <= r) F[pk(r, c, m)] = g[c];
    }
  }
  if (r < m) {
    vs[r] = vI;
    if (active) node_Y<T>(a.arenas, nd, s)[r] = vI;
  }
  const int g_elems = m * (m + 1) / 2;
  if (active)
    for (int i = r; i < b; i += 16) F[g_elems + i] = wv[i];
  __syncwarp();
  if (!active) return;

  // 4. lower Schur triangle ((b+1) x (b+1), column-major), walked in packed order
  T* S = leaf_S<T>(a.arenas, nd, s);
  const int total = nb * (nb + 1) / 2;
  int c = 0, off = r;   // entry (c + off, c)
  while (c < nb && off >= nb - c) { off -= nb - c; ++c; }
  for (int t = r; t < total; t += 16) {
    const int i = c + off, j = c;   // i >= j
    T val = (T)0;
    if (i < b) {
      val = (i == j) ? dB[i] : ((nj0[i] == j) ? nw0[i] : ((nj1[i] == j) ? nw1[i] : (T)0));
      const int ci = cpl[i], cj = cpl[j];
      if (ci >= 0 && cj >= 0) val -= wv[i] * wv[j] * Gs[ci * kLd + cj];
    } else if (j < b) {   // condensed load (bordered row)
      const int cj = cpl[j];
      if (cj >= 0) val = -wv[j] * vs[cj];
    }
    S[j * nb + i] = val;
    off += 16;
    while (c < nb && off >= nb - c) { off -= nb - c; ++c; }
  }
}

// Right-hand-side sweep at condensed leaves: y_g = G r_g, z_B,i = -w_i y_g[c_i]
// (written to the start of the leaf's Schur block, where the father reads it).
// One half-warp per (leaf, sample), lane r = interior row r.
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_forward(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, Arenas A,
                                                      Rhs rhs) {
  const int node = list[blockIdx.x];
  const int hw = threadIdx.x >> 4, r = threadIdx.x & 15;
  const int s = blockIdx.y * kLeafSamples + hw;
  const bool active = s < batch;   // both half-warps stay for the shuffles
  const int ss = active ? s : 0;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const T* F = leaf_F<T>(A, nd, ss);
  const T z = (r < m) ? (T)rhs(ss, vid[r]) : (T)0;
  T v = (T)0;
#pragma unroll
  for (int j = 0; j < kLeafInvMax; ++j) {
    const T zj = __shfl_sync(kAllLanes, z, j, 16);
    if (r < m && j < m) v += F[r >= j ? pk(r, j, m) : pk(j, r, m)] * zj;
  }
  if (active && r < m) node_Y<T>(A, nd, s)[r] = v;
  T* S = leaf_S<T>(A, nd, ss);
  const int g_elems = m * (m + 1) / 2;
  for (int i0 = 0; i0 < b; i0 += 16) {
    const int i = i0 + r;
    const int ci = (i < b) ? cpl[i] : -1;
    const T vc = __shfl_sync(kAllLanes, v, ci >= 0 ? ci : 0, 16);
    if (active && i < b) S[i] = (ci >= 0) ? -F[g_elems + i] * vc : (T)0;
  }
}

// Descent at condensed leaves: u_g = y_g - sum_i (w_i u_B,i) G[:, c_i].  One
// half-warp per (leaf, sample).
template <typename T>
__global__ void __launch_bounds__(256) k_leaf_descent(const NodeDev* __restrict__ nodes,
                                                      const int32_t* __restrict__ maps,
                                                      const int32_t* __restrict__ list, int batch, Arenas A,
                                                      double* __restrict__ u, int64_t u_stride) {
  const int node = list[blockIdx.x];
  const int hw = threadIdx.x >> 4, r = threadIdx.x & 15;
  const int s = blockIdx.y * kLeafSamples + hw;
  const bool active = s < batch;
  const int ss = active ? s : 0;
  __shared__ T tw[kLeafSamples][kLeafInvMaxB + 1];
  __shared__ int cw[kLeafSamples][kLeafInvMaxB + 1];
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const int32_t* vid = maps + nd.map_off;
  const int32_t* cpl = vid + (nf - 1);
  const T* F = leaf_F<T>(A, nd, ss);
  double* us = u + (int64_t)ss * u_stride;
  const int g_elems = m * (m + 1) / 2;
  for (int i = r; i < b; i += 16) {
    cw[hw][i] = cpl[i];
    tw[hw][i] = F[g_elems + i] * (T)us[vid[m + i]];
  }
  __syncwarp();
  if (r < m) {
    T acc = node_Y<T>(A, nd, ss)[r];
    for (int i = 0; i < b; ++i) {
      const int ci = cw[hw][i];
      if (ci >= 0) acc -= tw[hw][i] * F[r >= ci ? pk(r, ci, m) : pk(ci, r, m)];
    }
    if (active) us[vid[r]] = (double)acc;
  }
}

template <typename T>
cudaError_t launch_leaf_front(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  const size_t smem = (size_t)kLeafSamples * (samp_elems<T>() * sizeof(T) + kSampInts * sizeof(int)) +
                      (size_t)(a.max_rect + a.max_nf) * sizeof(int);
  if (a.prof) a.prof->begin(kProfLeaf, a.fl_chol + a.fl_trsm + a.fl_syrk + a.fl_rhs, st);
  k_leaf_front<T><<<dim3(a.nlist, (a.batch + kLeafSamples - 1) / kLeafSamples), 256, smem, st>>>(a);
  if (a.prof) a.prof->end(st);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_leaf_forward(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, const Rhs& rhs, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_leaf_forward<T><<<dim3(nlist, (batch + kLeafSamples - 1) / kLeafSamples), 256, 0, st>>>(nodes, maps, list, batch,
                                                                                            A, rhs);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_leaf_descent(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                                const Arenas& A, double* u, int64_t u_stride, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  k_leaf_descent<T><<<dim3(nlist, (batch + kLeafSamples - 1) / kLeafSamples), 256, 0, st>>>(nodes, maps, list, batch,
                                                                                            A, u, u_stride);
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
