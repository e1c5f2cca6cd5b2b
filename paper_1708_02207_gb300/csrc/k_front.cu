// Front kernels of the upsweep ("Leaves to Root", Sec. 3.4).
//
// A front of node omega is the matrix of the local system over
// [gamma (m rows), boundary unknowns (b rows), right-hand side (1 row)]:
//   leaves  - the stiffness of the leaf's own triangles (Sec. 3.1, Eq. coefA), load
//             at the interior rows (Eq. coefc);
//   fathers - the sons' Schur complements added into the union of their
//             boundaries (Sec. 3.3, Eq. block_equation4) plus the load of gamma.
// Eliminating gamma by a partial Cholesky gives the Schur maps of Sec. 2.4
// (Eq. SchurC1): L_gg L_gg^T = K_gg, L_Bg = K_Bg L_gg^-T, S = K_BB - L_Bg L_Bg^T;
// the bordered right-hand-side row turns into y_g^T = (L_gg^-1 b_g)^T and the
// condensed load b_B - L_Bg y_g, i.e. Psi^f c of the paper.
#include "launch.h"

namespace hdd {

template <typename T> __device__ __forceinline__ T* node_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* node_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* node_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* node_S(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* node_S<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* node_S<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

__device__ __forceinline__ double front_entry(int r, int c, int s, int node, const NodeDev& nd,
                                              const NodeDev* nodes, const int32_t* map, const double* kap,
                                              int N, const Rhs& rhs, const Arenas& A) {
  if (nd.leaf) return leaf_entry(r, c, s, nd, map, kap, N, rhs);
  return father_entry(r, c, s, nd, map, nodes[nd.child0], nodes[nd.child1], A, rhs);
}

// ---------------------------------------------------------------------------
// Fronts of 33..kSmallMax rows: the whole front lives in shared memory
// (column-major, ld nf), one CTA per (node, sample).  Fathers are assembled by
// scattering each son's lower Schur triangle (read column by column, coalesced)
// through the son's up map; sons one after the other, then the gamma loads.
// Partial Cholesky: per column k, scale column k, then one warp per trailing
// column j updates rows j..nf-1 (contiguous, conflict-free) with l_j.
template <typename T>
__device__ __forceinline__ void scatter_son(T* K, int nf, const NodeDev& ch, const int32_t* maps, const Arenas& A,
                                            int s) {
  const int ldc = ch.b + 1;
  const int32_t* up = maps + ch.up_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int64_t base = (int64_t)s * (ch.fp64 ? A.s64_stride : A.s32_stride) + ch.s_off;
  for (int cc = warp; cc < ldc; cc += nwarp) {
    const int pc = up[cc];
    for (int aa = cc + lane; aa < ldc; aa += 32) {
      const int64_t idx = base + (int64_t)cc * ldc + aa;
      const T val = ch.fp64 ? (T)A.s64[idx] : (T)A.s32[idx];
      const int pr = up[aa];
      const int r = max(pr, pc), c = min(pr, pc);
      K[c * nf + r] += val;
    }
  }
}

template <typename T>
__global__ void k_front_small(StepArgs a) {
  const int node = a.list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* K = reinterpret_cast<T*>(smem_raw);
  const int32_t* map = a.maps + nd.map_off;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;

  if (nd.leaf) {
    const double* kap = a.kappa + (int64_t)s * a.kap_stride;
    for (int idx = threadIdx.x; idx < nf * nf; idx += blockDim.x) {
      const int c = idx / nf, r = idx - c * nf;
      K[idx] = (r >= c) ? (T)leaf_entry(r, c, s, nd, map, kap, a.N, a.rhs) : (T)0;
    }
  } else {
    for (int idx = threadIdx.x; idx < nf * nf; idx += blockDim.x) K[idx] = (T)0;
    __syncthreads();
    scatter_son<T>(K, nf, a.nodes[nd.child0], a.maps, a.arenas, s);
    __syncthreads();
    scatter_son<T>(K, nf, a.nodes[nd.child1], a.maps, a.arenas, s);
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) K[c * nf + nf - 1] += (T)a.rhs(s, map[c]);
  }
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    T p = K[k * nf + k];
    if (!(p > (T)0) || !isfinite(p)) {   // not SPD: record, continue with a unit pivot
      if (threadIdx.x == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
      p = (T)1;
    }
    const T d = sqrt(p), inv = (T)1 / d;
    T* colk = K + k * nf;
    for (int i = k + 1 + threadIdx.x; i < nf; i += blockDim.x) colk[i] *= inv;
    __syncthreads();
    if (threadIdx.x == 0) colk[k] = d;
    for (int j = k + 1 + warp; j < nf; j += nwarp) {
      const T lj = colk[j];
      T* colj = K + j * nf;
      for (int i = j + lane; i < nf; i += 32) colj[i] -= colk[i] * lj;
    }
  }
  __syncthreads();
  T* F = node_F<T>(a.arenas, nd, s);
  for (int idx = threadIdx.x; idx < m * nf; idx += blockDim.x) F[idx] = K[idx];
  const int nb = nd.b + 1;
  T* S = node_S<T>(a.arenas, nd, s);
  for (int c = warp; c < nb; c += nwarp)
    for (int r = c + lane; r < nb; r += 32) S[c * nb + r] = K[(m + c) * nf + m + r];
}

static int small_threads(int nf) { return nf <= 64 ? 128 : 256; }

template <typename T>
cudaError_t launch_front_small(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  const size_t smem = (size_t)a.max_nf * a.max_nf * sizeof(T);
  dim3 grid(a.nlist, a.batch);
  k_front_small<T><<<grid, small_threads(a.max_nf), smem, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Large fronts (global memory).  Fill: one warp per front column.
template <typename T>
__global__ void k_front_fill(StepArgs a) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  const NodeDev nd = a.nodes[node];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1;
  if (c >= nf) return;
  const int32_t* map = a.maps + nd.map_off;
  const double* kap = a.kappa + (int64_t)s * a.kap_stride;
  T* F = node_F<T>(a.arenas, nd, s);
  T* S = node_S<T>(a.arenas, nd, s);
  for (int r = lane; r < nf; r += 32) {
    const T v = (r >= c) ? (T)front_entry(r, c, s, node, nd, a.nodes, map, kap, a.N, a.rhs, a.arenas) : (T)0;
    if (c < m) F[(int64_t)c * nf + r] = v;
    else if (r >= m) S[(int64_t)(c - m) * nb + (r - m)] = v;
  }
}

// POTRF of K_gg (m x m, in F with ld nf): one CTA per (node, sample), blocked
// right-looking with 32-column panels staged in shared memory; the trailing
// update uses 4 x 4 register tiles over the lower triangle.
constexpr int kPanel = 32;

__device__ __forceinline__ void tri_index(int idx, int& ti, int& tj) {
  int t = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
  while (t * (t + 1) / 2 > idx) --t;
  while ((t + 1) * (t + 2) / 2 <= idx) ++t;
  ti = t;
  tj = idx - t * (t + 1) / 2;
}

// Rows of a panel (POTRF) or of a row block (TRSM) kept in shared memory; larger
// fronts work in place in global memory through the same indexing.
template <typename T> struct SmemCap;
template <> struct SmemCap<double> { static constexpr int rows = 800; };
template <> struct SmemCap<float> { static constexpr int rows = 1600; };

template <typename T>
__global__ void k_potrf(StepArgs a) {
  const int node = a.list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* piv = reinterpret_cast<T*>(smem_raw);                 // [kPanel]
  T* Ps = piv + kPanel;                                     // panel, ld = rows
  const bool in_smem = m <= SmemCap<T>::rows;
  for (int k0 = 0; k0 < m; k0 += kPanel) {
    const int kb = min(kPanel, m - k0), rows = m - k0;
    T* P = in_smem ? Ps : A + (int64_t)k0 * nf + k0;
    const int ld = in_smem ? rows : nf;
    __syncthreads();
    if (in_smem)
      for (int idx = threadIdx.x; idx < kb * rows; idx += blockDim.x) {
        const int l = idx / rows, i = idx - l * rows;
        Ps[idx] = A[(int64_t)(k0 + l) * nf + k0 + i];
      }
    // factor the panel (rows k0..m-1, columns k0..k0+kb-1)
    for (int kk = 0; kk < kb; ++kk) {
      __syncthreads();
      T p = P[(int64_t)kk * ld + kk];
      if (!(p > (T)0) || !isfinite(p)) {
        if (threadIdx.x == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
        p = (T)1;
      }
      if (threadIdx.x == 0) piv[kk] = sqrt(p);
      const T rp = (T)1 / p;
      const T* colk = P + (int64_t)kk * ld;
      const int ncol = kb - kk - 1;                 // panel columns right of kk
      const int nrow = rows - kk - 1;               // rows below kk
      for (int idx = threadIdx.x; idx < ncol * nrow; idx += blockDim.x) {
        const int jj = idx / nrow, ii = idx - jj * nrow;
        if (ii < jj) continue;
        const int i = kk + 1 + ii, j = kk + 1 + jj;
        P[(int64_t)j * ld + i] -= colk[i] * (colk[j] * rp);
      }
      if (kk > 0) {
        const int c = kk - 1;
        const T d = piv[c], rd = (T)1 / d;
        for (int i = c + threadIdx.x; i < rows; i += blockDim.x)
          P[(int64_t)c * ld + i] = (i == c) ? d : P[(int64_t)c * ld + i] * rd;
      }
    }
    __syncthreads();
    {
      const int c = kb - 1;
      const T d = piv[c], rd = (T)1 / d;
      for (int i = c + threadIdx.x; i < rows; i += blockDim.x)
        P[(int64_t)c * ld + i] = (i == c) ? d : P[(int64_t)c * ld + i] * rd;
    }
    __syncthreads();
    if (in_smem)
      for (int idx = threadIdx.x; idx < kb * rows; idx += blockDim.x) {
        const int l = idx / rows, i = idx - l * rows;
        if (i >= l) A[(int64_t)(k0 + l) * nf + k0 + i] = Ps[idx];
      }
    // trailing update of K_gg[k0+kb:m, k0+kb:m] (lower)
    const int n = rows - kb;
    if (n <= 0) continue;
    const int nt = (n + 3) / 4;
    const int ntiles = nt * (nt + 1) / 2;
    for (int idx = threadIdx.x; idx < ntiles; idx += blockDim.x) {
      int ti, tj;
      tri_index(idx, ti, tj);
      const int i0 = kb + 4 * ti, j0 = kb + 4 * tj;   // panel-relative rows
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
      for (int l = 0; l < kb; ++l) {
        T x[4], y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          x[q] = (i0 + q < rows) ? P[(int64_t)l * ld + i0 + q] : (T)0;
          y[q] = (j0 + q < rows) ? P[(int64_t)l * ld + j0 + q] : (T)0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int j = j0 + w;
        if (j >= rows) break;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + q;
          if (i < rows && i >= j) A[(int64_t)(k0 + j) * nf + k0 + i] -= acc[q][w];
        }
      }
    }
  }
}

// TRSM: rows m..nf-1 of F times L_gg^-T.  One CTA per (32-row block, node, sample);
// the block's rows stay in shared memory across the column sweep.
constexpr int kTrsmRows = 32;

template <typename T>
__global__ void k_trsm(StepArgs a) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  const int r0 = m + blockIdx.x * kTrsmRows;
  if (r0 >= nf || m == 0) return;
  const int nr = min(kTrsmRows, nf - r0);
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);        // [32][33]
  T* Xs = L + 32 * 33;                          // [m][kTrsmRows]
  const bool in_smem = m <= SmemCap<T>::rows;
  // X(r, c) = X[c * ldx + r]: the row block in shared memory, or in place in F
  T* X = in_smem ? Xs : A + r0;
  const int64_t ldx = in_smem ? kTrsmRows : nf;
  if (in_smem)
    for (int idx = threadIdx.x; idx < m * kTrsmRows; idx += blockDim.x) {
      const int c = idx / kTrsmRows, r = idx - c * kTrsmRows;
      Xs[idx] = (r < nr) ? A[(int64_t)c * nf + r0 + r] : (T)0;
    }
  const int r = threadIdx.x % kTrsmRows, grp = threadIdx.x / kTrsmRows, ngrp = blockDim.x / kTrsmRows;
  const bool row_ok = r < nr;
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int jb = min(32, m - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < jb * jb; idx += blockDim.x) {
      const int l = idx / jb, q = idx - l * jb;
      L[l * 33 + q] = (q >= l) ? A[(int64_t)(j0 + l) * nf + j0 + q] : (T)0;
    }
    __syncthreads();
    if (threadIdx.x < kTrsmRows && row_ok) {
      for (int cc = 0; cc < jb; ++cc) {
        T x = X[(j0 + cc) * ldx + r];
        for (int l = 0; l < cc; ++l) x -= X[(j0 + l) * ldx + r] * L[l * 33 + cc];
        X[(j0 + cc) * ldx + r] = x / L[cc * 33 + cc];
      }
    }
    __syncthreads();
    if (row_ok)
      for (int c2 = j0 + jb + grp; c2 < m; c2 += ngrp) {
        T acc = (T)0;
        for (int l = 0; l < jb; ++l) acc += X[(j0 + l) * ldx + r] * A[(int64_t)(j0 + l) * nf + c2];
        X[c2 * ldx + r] -= acc;
      }
  }
  __syncthreads();
  if (in_smem)
    for (int idx = threadIdx.x; idx < m * kTrsmRows; idx += blockDim.x) {
      const int c = idx / kTrsmRows, rr = idx - c * kTrsmRows;
      if (rr < nr) A[(int64_t)c * nf + r0 + rr] = Xs[idx];
    }
}

// SYRK: S -= X X^T with X = F[m:nf, 0:m] (b+1 rows incl. the right-hand side).
// One CTA per (64 x 64 lower tile pair, node, sample), 4 x 4 per thread.
constexpr int kSyrkTile = 64, kSyrkK = 16;

template <typename T>
__global__ void k_syrk(StepArgs a) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1;
  const int nt = (nb + kSyrkTile - 1) / kSyrkTile;
  if ((int)blockIdx.x >= nt * (nt + 1) / 2 || m == 0) return;
  int TI, TJ;
  tri_index(blockIdx.x, TI, TJ);
  const T* X = node_F<T>(a.arenas, nd, s) + m;
  T* S = node_S<T>(a.arenas, nd, s);
  __shared__ T As[kSyrkK][kSyrkTile], Bs[kSyrkK][kSyrkTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
  for (int k0 = 0; k0 < m; k0 += kSyrkK) {
    const int kc = min(kSyrkK, m - k0);
    for (int e = threadIdx.x; e < kSyrkK * kSyrkTile; e += blockDim.x) {
      const int kk = e / kSyrkTile, ii = e - kk * kSyrkTile;
      const int ri = TI * kSyrkTile + ii, rj = TJ * kSyrkTile + ii;
      As[kk][ii] = (kk < kc && ri < nb) ? X[(int64_t)(k0 + kk) * nf + ri] : (T)0;
      Bs[kk][ii] = (kk < kc && rj < nb) ? X[(int64_t)(k0 + kk) * nf + rj] : (T)0;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      T x[4], y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { x[q] = As[kk][ty + 16 * q]; y[q] = Bs[kk][tx + 16 * q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = TI * kSyrkTile + ty + 16 * q;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int j = TJ * kSyrkTile + tx + 16 * w;
      if (i < nb && j < nb && i >= j) S[(int64_t)j * nb + i] -= acc[q][w];
    }
  }
}

template <typename T>
cudaError_t launch_front_large(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  {
    dim3 grid((a.max_nf + 7) / 8, a.nlist, a.batch);
    k_front_fill<T><<<grid, 256, 0, st>>>(a);
  }
  const size_t rows_smem = (size_t)min(a.max_m, SmemCap<T>::rows);
  {
    const size_t smem = (rows_smem * kPanel + kPanel) * sizeof(T);
    k_potrf<T><<<dim3(a.nlist, a.batch), 256, smem, st>>>(a);
  }
  {
    const size_t smem = (rows_smem * kTrsmRows + 32 * 33) * sizeof(T);
    dim3 grid((a.max_b + 1 + kTrsmRows - 1) / kTrsmRows, a.nlist, a.batch);
    k_trsm<T><<<grid, 256, smem, st>>>(a);
  }
  {
    const int nt = (a.max_b + 1 + kSyrkTile - 1) / kSyrkTile;
    dim3 grid(nt * (nt + 1) / 2, a.nlist, a.batch);
    k_syrk<T><<<grid, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

template cudaError_t launch_front_small<double>(const StepArgs&, cudaStream_t);
template cudaError_t launch_front_small<float>(const StepArgs&, cudaStream_t);
template cudaError_t launch_front_large<double>(const StepArgs&, cudaStream_t);
template cudaError_t launch_front_large<float>(const StepArgs&, cudaStream_t);

cudaError_t configure_front_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_front_small<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_front_small<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
