// Large-front kernels of the upsweep ("Leaves to Root", Sec. 3.4).
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
#include <type_traits>

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

// Panel width of the blocked POTRF of large fronts.
constexpr int kPanel = 32;

__device__ __forceinline__ void tri_index(int idx, int& ti, int& tj) {
  int t = (int)((sqrtf(8.0f * (float)idx + 1.0f) - 1.0f) * 0.5f);
  while (t * (t + 1) / 2 > idx) --t;
  while ((t + 1) * (t + 2) / 2 <= idx) ++t;
  ti = t;
  tj = idx - t * (t + 1) / 2;
}

// Four consecutive values through 16-byte shared-memory accesses.
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// ---------------------------------------------------------------------------
// Large fronts (global memory).  Fill: one warp per front column, columns
// 0..ncols-1 (all nf columns, or only the m gamma columns when the Schur
// update gathers the sons' entries itself).  Father entries are gathered from
// the sons' lower Schur triangles through the position maps (son row of each
// front row, -1 if absent), with the column's positions hoisted and four rows
// per lane loaded before any store.
template <typename T, typename TS>
__device__ __forceinline__ void fill_father_column(T* F, T* S, int c, int lane, const NodeDev& nd, const int32_t* map,
                                                   const TS* S0, int ld0, const TS* S1, int ld1, T load_c) {
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1;
  const int32_t* pos0 = map + (nf - 1);
  const int32_t* pos1 = pos0 + nf;
  const int q0 = pos0[c], q1 = pos1[c];
  if (c < m)
    for (int r = lane; r < c; r += 32) F[(int64_t)c * nf + r] = (T)0;
  for (int r0 = c + lane; r0 < nf; r0 += 128) {
    T v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + 32 * q;
      v[q] = (T)0;
      if (r < nf) {
        const int a0 = pos0[r], a1 = pos1[r];
        if (a0 >= 0 && q0 >= 0) v[q] += (T)S0[min(a0, q0) * ld0 + max(a0, q0)];
        if (a1 >= 0 && q1 >= 0) v[q] += (T)S1[min(a1, q1) * ld1 + max(a1, q1)];
        if (r == nf - 1) v[q] += load_c;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + 32 * q;
      if (r >= nf) break;
      if (c < m) F[(int64_t)c * nf + r] = v[q];
      else if (r >= m) S[(int64_t)(c - m) * nb + (r - m)] = v[q];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_front_fill(StepArgs a, int gamma_only) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1;
  if (c >= ((gamma_only && !nd.leaf) ? m : nf)) return;   // leaves fill their whole front
  const int32_t* map = a.maps + nd.map_off;
  T* F = node_F<T>(a.arenas, nd, s);
  T* S = node_S<T>(a.arenas, nd, s);
  if (nd.leaf) {
    const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)s * a.kap_stride;
    for (int r = lane; r < nf; r += 32) {
      const T v = (r >= c) ? leaf_entry<T>(r, c, s, nd, map, kap, a.N, a.rhs) : (T)0;
      if (c < m) F[(int64_t)c * nf + r] = v;
      else if (r >= m) S[(int64_t)(c - m) * nb + (r - m)] = v;
    }
    return;
  }
  const NodeDev c0 = a.nodes[nd.child0], c1 = a.nodes[nd.child1];
  const T load_c = (c < m) ? (T)a.rhs(s, map[c]) : (T)0;
  const Arenas& A = a.arenas;
  if (!c0.fp64 && !c1.fp64)
    fill_father_column<T, float>(F, S, c, lane, nd, map, A.s32 + (int64_t)s * A.s32_stride + c0.s_off, c0.b + 1,
                                 A.s32 + (int64_t)s * A.s32_stride + c1.s_off, c1.b + 1, load_c);
  else if (c0.fp64 && c1.fp64)
    fill_father_column<T, double>(F, S, c, lane, nd, map, A.s64 + (int64_t)s * A.s64_stride + c0.s_off, c0.b + 1,
                                  A.s64 + (int64_t)s * A.s64_stride + c1.s_off, c1.b + 1, load_c);
  else
    for (int r = lane; r < nf; r += 32) {
      const T v = (r >= c) ? father_entry<T>(r, c, s, nd, map, c0, c1, A, a.rhs) : (T)0;
      if (c < m) F[(int64_t)c * nf + r] = v;
      else if (r >= m) S[(int64_t)(c - m) * nb + (r - m)] = v;
    }
}

// Rows of a panel (POTRF) or of a row block (TRSM) kept in shared memory; larger
// fronts work in place in global memory through the same indexing.
template <typename T> struct SmemCap;
template <> struct SmemCap<double> { static constexpr int rows = 800; };
template <> struct SmemCap<float> { static constexpr int rows = 1600; };

// Staging for the tensor-core SYRK (k_syrk_tc): rows [row0, row0 + nr) of X
// (= F[m:nf, 0:m], relative row numbers; the bordered right-hand-side row is
// excluded, k_syrk_rhs handles it) split into TF32 hi and lo parts and written in
// 128-row x kTcChunk-column tiles, K-major core-matrix layout (8 rows x 16 bytes
// per core matrix, cores along K 128 bytes apart).  The block holding the last
// boundary row also zero-fills the rest of its tile.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void write_tc_tiles(const float* X, int64_t ldx, const NodeDev& nd, const Arenas& A, int s,
                                               int row0, int nr, bool last) {
  if (nd.b == 0) return;
  const int m = nd.m;
  const int nchunks = (m + kTcChunk - 1) / kTcChunk;
  if (last) --nr;                      // the right-hand-side row
  if (last && nr == 0 && row0 % kTcTile == 0) return;   // nothing of this tile is a boundary row
  const int rows = last ? ((row0 / kTcTile) + 1) * kTcTile - row0 : nr;   // zero-fill to the tile end
  unsigned char* base = A.tc + (int64_t)s * A.tc_stride + nd.tc_off;
  const int items = rows * nchunks * (kTcChunk / 4);
  for (int idx = threadIdx.x; idx < items; idx += blockDim.x) {
    const int rr = idx % rows;
    const int rest = idx / rows;
    const int kq = rest % (kTcChunk / 4), c = rest / (kTcChunk / 4);
    const int row = row0 + rr, T = row / kTcTile, tr = row % kTcTile;
    float v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = c * kTcChunk + 4 * kq + q;
      v[q] = (rr < nr && k < m) ? X[(int64_t)k * ldx + rr] : 0.0f;
    }
    float4 hi, lo;
    hi.x = tf32_rna(v[0]); hi.y = tf32_rna(v[1]); hi.z = tf32_rna(v[2]); hi.w = tf32_rna(v[3]);
    lo.x = tf32_rna(v[0] - hi.x); lo.y = tf32_rna(v[1] - hi.y); lo.z = tf32_rna(v[2] - hi.z); lo.w = tf32_rna(v[3] - hi.w);
    const int64_t blk = ((int64_t)T * nchunks + c) * 2 * kTcBlockBytes;
    const int off = (tr >> 3) * (kTcChunk / 4) * 128 + kq * 128 + (tr & 7) * 16;
    *reinterpret_cast<float4*>(base + blk + off) = hi;
    *reinterpret_cast<float4*>(base + blk + kTcBlockBytes + off) = lo;
  }
}

// TRSM: rows m..nf-1 of F times L_gg^-T.  One CTA per (row block, node, sample);
// the row block X stays in shared memory across the column sweep (or is updated
// in place in global memory when m is too large).  Per 32-column block of L_gg:
// the diagonal triangle is solved one thread per row, then the remaining columns
// are updated in 64-column chunks of L staged in shared memory, with register
// micro-tiles (4 rows x kTrsmCols columns per thread).
// POTRF and TRSM of large fronts whose gamma block has at most 32 * NB columns
// (NB = 1, 2), one CTA per (node, sample).  Diagonal 32 x 32 blocks are factored
// by warp 0 in registers (pivot column by shuffles) and inverted in shared
// memory (lane c solves L w = e_c); for NB = 2 the block below the first
// diagonal block is L21 = A21 W11^T and the second diagonal block is factored
// after A22 - L21 L21^T.  Every thread then takes boundary rows, their gamma
// entries in registers, and applies the blocked substitution
//   x_0 = a_0 W11^T,  x_1 = (a_1 - x_0 L21^T) W22^T
// (the same arithmetic as k_potrf + k_trsm), writing the factor rows, y_g
// (bordered row) and, for FP32 fronts, the split TF32 tiles of the
// tensor-core Schur update.
constexpr int kWs = 36;   // row stride of shared 32 x 32 blocks read four columns at a time

// Cholesky of the 32 x 32 block held as rows (lane r: row r, entries c <= r; size
// mb), its inverse into W (W[r][c] at W[r * kWs + c]); L itself into Ls.
template <typename T>
__device__ __forceinline__ void warp_chol_inverse(T (&row)[32], int mb, T* Ls, T* W, T* dinv, bool& bad) {
  constexpr unsigned kAll = 0xffffffffu;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < mb) {
      T pk = __shfl_sync(kAll, row[k], k);
      if (!(pk > (T)0) || !isfinite(pk)) {
        bad = true;
        pk = (T)1;
      }
      const T d = sqrt(pk), inv = (T)1 / d;
      T lk = (lane == k) ? d : row[k] * inv;
      if (lane < k) lk = (T)0;
#pragma unroll
      for (int j = k + 1; j < 32; ++j) {
        const T lj = __shfl_sync(kAll, lk, j);
        if (lane > k) row[j] -= lk * lj;
      }
      row[k] = lk;
    }
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) Ls[lane * kWs + c] = row[c];
  T diag = (T)1;
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (c == lane && c < mb) diag = row[c];
  dinv[lane] = (T)1 / diag;
  __syncwarp();
  T w[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    T acc = (lane == r) ? (T)1 : (T)0;
#pragma unroll
    for (int l = 0; l < r; ++l) acc -= Ls[r * kWs + l] * w[l];
    w[r] = (r < mb) ? acc * dinv[r] : (T)0;
    W[r * kWs + lane] = (lane < mb) ? w[r] : (T)0;
  }
}

// x <- x W^T in place for the 32 entries x[o .. o+31] (W lower, last column first)
template <typename T, int O, int NX>
__device__ __forceinline__ void apply_inverse(T (&x)[NX], const T* W) {
#pragma unroll
  for (int c = 31; c >= 0; --c) {
    T acc = (T)0;
#pragma unroll
    for (int l4 = 0; l4 <= c; l4 += 4) {
      T wv[4];
      load4(W + c * kWs + l4, wv);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (l4 + q <= c) acc += x[O + l4 + q] * wv[q];
    }
    x[O + c] = acc;
  }
}

// POTRF of K_gg (m x m, in F with ld nf): one CTA per (node, sample), blocked
// right-looking with 32-column panels staged in shared memory.  Per panel, warp 0
// factors the 32 x 32 diagonal block in registers and inverts it
// (warp_chol_inverse: the pivot column by shuffles, no CTA barrier per column);
// the panel rows below it become L21 = A21 L11^-T as products with that inverse,
// one thread per row; the trailing update uses 4 x 4 register tiles over the
// lower triangle.  The inverse also goes to the arena of inverted diagonal blocks,
// which the TRSM applies as products.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_potrf(StepArgs a) {   // FP64 panels fill the shared memory
  const int node = a.list[blockIdx.x];
  const int s = blockIdx.y;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);   // [32][kWs] scratch of warp_chol_inverse
  T* W = Ls + 32 * kWs;                     // [32][kWs] inverse of the diagonal block, W[r * kWs + c]
  T* dinv = W + 32 * kWs;                   // [32]
  T* Ps = dinv + 32;                        // panel, ld = rows rounded up to 4 (16 B aligned)
  const bool in_smem = m <= SmemCap<T>::rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  bool bad = false;
  for (int k0 = 0; k0 < m; k0 += kPanel) {
    const int kb = min(kPanel, m - k0), rows = m - k0;
    T* P = in_smem ? Ps : A + (int64_t)k0 * nf + k0;
    const int ld = in_smem ? ((rows + 3) & ~3) : nf;
    __syncthreads();
    if (in_smem)   // one warp per panel column, eight rows per lane in flight
      for (int l = warp; l < kb; l += nwarp)
        for (int i0 = lane; i0 < rows; i0 += 256) {
          T v[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = i0 + 32 * q;
            v[q] = i < rows ? A[(int64_t)(k0 + l) * nf + k0 + i] : (T)0;
          }
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (i0 + 32 * q < rows) Ps[l * ld + i0 + 32 * q] = v[q];
        }
    __syncthreads();
    if (warp == 0) {   // the diagonal block, lane r holding row r
      T row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = (c < kb && lane < kb && c <= lane) ? P[(int64_t)c * ld + lane] : (T)0;
      warp_chol_inverse<T>(row, kb, Ls, W, dinv, bad);
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < kb && lane < kb && c <= lane) P[(int64_t)c * ld + lane] = row[c];
      // column c of the inverse at G[c * 32 .. c * 32 + 31] (identity beyond the block)
      T* G = reinterpret_cast<T*>(a.arenas.inv + (int64_t)s * a.arenas.inv_stride + nd.inv_off) + (k0 / 32) * 1024;
#pragma unroll 4
      for (int r = 0; r < 32; ++r)
        G[lane * 32 + r] = (lane < kb) ? ((r < kb) ? W[r * kWs + lane] : (T)0) : ((r == lane) ? (T)1 : (T)0);
    }
    __syncthreads();
    // rows below the diagonal block (present only for full panels, kb = 32): x <- x W^T
    for (int i = kb + threadIdx.x; i < rows; i += blockDim.x) {
      T x[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) x[l] = P[(int64_t)l * ld + i];
      apply_inverse<T, 0, 32>(x, W);
#pragma unroll
      for (int c = 0; c < 32; ++c) P[(int64_t)c * ld + i] = x[c];
    }
    __syncthreads();
    if (in_smem)
      for (int l = warp; l < kb; l += nwarp)
        for (int i = l + lane; i < rows; i += 32) A[(int64_t)(k0 + l) * nf + k0 + i] = Ps[l * ld + i];
    // trailing update of K_gg[k0+kb:m, k0+kb:m] (lower): 4 x 4 register tiles,
    // one warp per column of tiles, lanes down the rows (coalesced in global memory)
    const int n = rows - kb;
    if (n <= 0) continue;
    const int nt = (n + 3) >> 2;
    for (int tj = warp; tj < nt; tj += nwarp) {
      const int j0 = kb + 4 * tj;
      for (int ti = tj + lane; ti < nt; ti += 32) {
        const int i0 = kb + 4 * ti;
        T acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
        for (int l = 0; l < kb; ++l) {
          T x[4], y[4];
          if (in_smem) {   // kb = 32 here (a trailing block exists), so i0, j0 and ld are multiples of 4;
                           // the padding rows beyond `rows` only reach products that are not stored
            load4(P + l * ld + i0, x);
            load4(P + l * ld + j0, y);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              x[q] = (i0 + q < rows) ? P[(int64_t)l * ld + i0 + q] : (T)0;
              y[q] = (j0 + q < rows) ? P[(int64_t)l * ld + j0 + q] : (T)0;
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
        }
        T av[4][4];   // loads first (in flight together), then the stores
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + w, i = i0 + q;
            av[q][w] = (j < rows && i < rows && i >= j) ? A[(int64_t)(k0 + j) * nf + k0 + i] : (T)0;
          }
#pragma unroll
        for (int w = 0; w < 4; ++w)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int j = j0 + w, i = i0 + q;
            if (j < rows && i < rows && i >= j) A[(int64_t)(k0 + j) * nf + k0 + i] = av[q][w] - acc[q][w];
          }
      }
    }
  }
  if (bad && threadIdx.x == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
}

// POTRF of a K_gg whose whole lower triangle fits in shared memory: the same
// blocked algorithm as k_potrf, with the trailing updates in shared memory (one
// load of the triangle, one store of the factor).  Storage: column j holds rows
// floor4(j) .. m4-1 (m4 = m rounded up to 4), columns packed one after another, so
// that every 4-row group starts on a 16-byte boundary:
//   (i, j) -> tri_off(j, m4) + i - floor4(j),
//   tri_off(j, m4) = 4 q m4 - 8 q (q - 1) + r (m4 - 4 q),  j = 4 q + r.
__host__ __device__ __forceinline__ int tri_off(int j, int m4) {
  const int q = j >> 2, r = j & 3;
  return 4 * q * m4 - 8 * q * (q - 1) + r * (m4 - 4 * q);
}
__host__ __device__ __forceinline__ int tri_elems(int m) {
  const int m4 = (m + 3) & ~3;
  return tri_off(m4, m4);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_potrf_smem(StepArgs a) {
  const int node = a.list[blockIdx.x];
  const int s = blockIdx.y;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m, m4 = (m + 3) & ~3;
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);   // [32][kWs] scratch of warp_chol_inverse
  T* W = Ls + 32 * kWs;                     // [32][kWs] inverse of the diagonal block
  T* dinv = W + 32 * kWs;                   // [32]
  T* P = dinv + 32;                         // the lower triangle, 16-byte aligned 4-row groups
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  auto at = [&](int i, int j) -> T& { return P[tri_off(j, m4) + i - (j & ~3)]; };
  // load: column by column, one warp per column, zeros above the diagonal and below m;
  // two columns' rows per pass, all loads in flight before the stores
  for (int j0 = warp; j0 < m; j0 += 2 * nwarp) {
    T v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + h * nwarp;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = (j & ~3) + lane + 32 * k;
        v[h][k] = (j < m && i >= j && i < m) ? A[(int64_t)j * nf + i] : (T)0;
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = j0 + h * nwarp;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = (j & ~3) + lane + 32 * k;
        if (j < m && i < m4) at(i, j) = v[h][k];
      }
    }
  }
  bool bad = false;
  for (int k0 = 0; k0 < m; k0 += kPanel) {
    const int kb = min(kPanel, m - k0);
    __syncthreads();
    if (warp == 0) {   // the diagonal block, lane r holding row k0 + r
      T row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = (c < kb && lane < kb && c <= lane) ? at(k0 + lane, k0 + c) : (T)0;
      warp_chol_inverse<T>(row, kb, Ls, W, dinv, bad);
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < kb && lane < kb && c <= lane) at(k0 + lane, k0 + c) = row[c];
      T* G = reinterpret_cast<T*>(a.arenas.inv + (int64_t)s * a.arenas.inv_stride + nd.inv_off) + (k0 / 32) * 1024;
#pragma unroll 4
      for (int r = 0; r < 32; ++r)
        G[lane * 32 + r] = (lane < kb) ? ((r < kb) ? W[r * kWs + lane] : (T)0) : ((r == lane) ? (T)1 : (T)0);
    }
    __syncthreads();
    // rows below the diagonal block (full panels only): x <- x W^T
    for (int i = k0 + kb + threadIdx.x; i < m; i += blockDim.x) {
      T x[32];
#pragma unroll
      for (int l = 0; l < 32; ++l) x[l] = at(i, k0 + l);
      apply_inverse<T, 0, 32>(x, W);
#pragma unroll
      for (int c = 0; c < 32; ++c) at(i, k0 + c) = x[c];
    }
    __syncthreads();
    // trailing update of rows and columns k0+kb .. m4-1 in 4 x 4 tiles (rows past m
    // are zero and stay unused); one warp per column of tiles, lanes down the rows
    const int t0 = k0 + kb;   // a multiple of 32 whenever a trailing block exists
    if (t0 >= m) continue;
    const int nt = (m4 - t0) >> 2;
    for (int tj = warp; tj < nt; tj += nwarp) {
      const int j0 = t0 + 4 * tj;
      for (int ti = tj + lane; ti < nt; ti += 32) {
        const int i0 = t0 + 4 * ti;
        T acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
#pragma unroll 4
        for (int l = 0; l < 32; ++l) {
          T x[4], y[4];
          load4(&at(i0, k0 + l), x);
          load4(&at(j0, k0 + l), y);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          T v[4];
          load4(&at(i0, j0 + w), v);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (i0 + q >= j0 + w) at(i0 + q, j0 + w) = v[q] - acc[q][w];
        }
      }
    }
  }
  __syncthreads();
  for (int j = warp; j < m; j += nwarp)
    for (int i = j + lane; i < m; i += 32) A[(int64_t)j * nf + i] = at(i, j);
  if (bad && threadIdx.x == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
}

// Largest interface whose triangle, with the diagonal-block scratch, fits the shared
// memory of one CTA.
template <typename T>
static bool potrf_in_smem(int max_m, size_t* bytes) {
  *bytes = ((size_t)2 * 32 * kWs + 32 + tri_elems(max_m)) * sizeof(T);
  return *bytes <= 48 * 1024;   // larger triangles cost residency: measured slower
}

template <typename T, int NB>
struct CholTrsmSmem {   // per warp (sample)
  T W[NB][32 * kWs];
  T Ls[32 * kWs];
  T L21[NB > 1 ? 32 * kWs : 4];
  T dinv[32];
};
constexpr int kCholTrsmWarps = 4;   // samples of one node per CTA, one warp each

template <typename T, int NB>
__global__ void __launch_bounds__(32 * kCholTrsmWarps, 3) k_chol_trsm(StepArgs a) {
  const int node = a.list[blockIdx.x];
  bind_plan(a, node);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.y * kCholTrsmWarps + warp;
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m, b = nd.b;
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CholTrsmSmem<T, NB>& sm = reinterpret_cast<CholTrsmSmem<T, NB>*>(smem_raw)[warp];
  const int mb0 = min(32, m), mb1 = m - mb0;
  bool bad = false;
  {
    T row[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) row[c] = (c < mb0 && lane < mb0 && c <= lane) ? A[(int64_t)c * nf + lane] : (T)0;
    warp_chol_inverse<T>(row, mb0, sm.Ls, sm.W[0], sm.dinv, bad);
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < mb0 && lane < mb0 && c <= lane) A[(int64_t)c * nf + lane] = row[c];
  }
  __syncwarp();
  if (NB > 1) {
    {   // L21 = A21 W11^T (rows 32..m-1, lane = row)
      T x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = (lane < mb1) ? A[(int64_t)c * nf + 32 + lane] : (T)0;
      apply_inverse<T, 0, 32>(x, sm.W[0]);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        sm.L21[lane * kWs + c] = (lane < mb1) ? x[c] : (T)0;
        if (lane < mb1) A[(int64_t)c * nf + 32 + lane] = x[c];
      }
    }
    __syncwarp();
    {   // second diagonal block: A22 - L21 L21^T
      T row[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        T v = (T)0;
        if (c < mb1 && lane < mb1 && c <= lane) {
          T dot = (T)0;
#pragma unroll
          for (int l4 = 0; l4 < 32; l4 += 4) {
            T p[4], q[4];
            load4(sm.L21 + lane * kWs + l4, p);
            load4(sm.L21 + c * kWs + l4, q);
#pragma unroll
            for (int t = 0; t < 4; ++t) dot += p[t] * q[t];
          }
          v = A[(int64_t)(32 + c) * nf + 32 + lane] - dot;
        }
        row[c] = v;
      }
      __syncwarp();
      warp_chol_inverse<T>(row, mb1, sm.Ls, sm.W[NB - 1], sm.dinv, bad);
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < mb1 && lane < mb1 && c <= lane) A[(int64_t)(32 + c) * nf + 32 + lane] = row[c];
    }
    __syncwarp();
  }
  if (bad && lane == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
  const bool tc = std::is_same<T, float>::value && nd.tc_off >= 0 && b > 0;
  const int nchunks = (m + kTcChunk - 1) / kTcChunk;
  unsigned char* tcb = tc ? a.arenas.tc + (int64_t)s * a.arenas.tc_stride + nd.tc_off : nullptr;
  const int tc_rows = ((b + kTcTile - 1) / kTcTile) * kTcTile;   // boundary rows, zero-filled to the tile end
  for (int r = m + lane; r < m + max(tc ? tc_rows : 0, nf - m); r += 32) {
    const bool real = r < nf;
    T y[32 * NB];   // the row's gamma entries, overwritten by its factor row
#pragma unroll
    for (int c = 0; c < 32 * NB; ++c) y[c] = (c < m && real) ? A[(int64_t)c * nf + r] : (T)0;
    apply_inverse<T, 0, 32 * NB>(y, sm.W[0]);
    if (NB > 1) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {   // a_1 - x_0 L21^T
        T dot = (T)0;
#pragma unroll
        for (int l4 = 0; l4 < 32; l4 += 4) {
          T q[4];
          load4(sm.L21 + j * kWs + l4, q);
#pragma unroll
          for (int t = 0; t < 4; ++t) dot += y[l4 + t] * q[t];
        }
        y[(NB - 1) * 32 + j] -= dot;
      }
      apply_inverse<T, (NB - 1) * 32, 32 * NB>(y, sm.W[NB - 1]);
    }
    if (real) {
#pragma unroll
      for (int c = 0; c < 32 * NB; ++c)
        if (c < m) A[(int64_t)c * nf + r] = y[c];
      if (r == nf - 1) {
        T* Y = node_Y<T>(a.arenas, nd, s);
#pragma unroll
        for (int c = 0; c < 32 * NB; ++c)
          if (c < m) Y[c] = y[c];
      }
    }
    const int br = r - m;   // boundary row (tile row space); the bordered row is not a tile row
    if (tc && br < tc_rows) {   // rows b.. (the bordered row included) are zero tile rows
      const int Tt = br / kTcTile, tr = br % kTcTile;
      const bool zero = br >= b;
#pragma unroll
      for (int c8 = 0; c8 < 4 * NB; ++c8) {
        if (c8 >= nchunks) break;
#pragma unroll
        for (int kq = 0; kq < 2; ++kq) {
          float v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = (zero || c8 * 8 + 4 * kq + q >= m) ? 0.0f : (float)y[c8 * 8 + 4 * kq + q];
          float4 hi, lo;
          hi.x = tf32_rna(v[0]); hi.y = tf32_rna(v[1]); hi.z = tf32_rna(v[2]); hi.w = tf32_rna(v[3]);
          lo.x = tf32_rna(v[0] - hi.x); lo.y = tf32_rna(v[1] - hi.y);
          lo.z = tf32_rna(v[2] - hi.z); lo.w = tf32_rna(v[3] - hi.w);
          const int64_t blk = ((int64_t)Tt * nchunks + c8) * 2 * kTcBlockBytes;
          const int off = (tr >> 3) * (kTcChunk / 4) * 128 + kq * 128 + (tr & 7) * 16;
          *reinterpret_cast<float4*>(tcb + blk + off) = hi;
          *reinterpret_cast<float4*>(tcb + blk + kTcBlockBytes + off) = lo;
        }
      }
    }
  }
}

template <typename T> struct TrsmShape;
template <> struct TrsmShape<float> { static constexpr int rows = 32, cap = 760; };   // rows: measured best of 32/64/128
template <> struct TrsmShape<double> { static constexpr int rows = 32, cap = 760; };

template <typename T, int R>
__global__ void __launch_bounds__(256) k_trsm(StepArgs a) {   // R rows per CTA
  constexpr int RG = R / 4;                 // row groups of 4
  constexpr int CG = 256 / RG;              // column groups
  constexpr int CPT = 64 / CG;              // columns per thread in a 64-column chunk
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  const int r0 = m + blockIdx.x * R;
  if (r0 >= nf || m == 0) return;
  const int nr = min(R, nf - r0);
  T* A = node_F<T>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);    // [32][33] diagonal block
  T* Lc = L + 32 * 33 + 3;                  // [32][64] chunk of the panel below it
  Lc = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(Lc) + 15) & ~uintptr_t(15));
  T* Xs = Lc + 32 * 64;                     // [m][R]
  const bool in_smem = m <= TrsmShape<T>::cap;
  T* X = in_smem ? Xs : A + r0;
  const int64_t ldx = in_smem ? R : nf;
  if (in_smem)
    for (int i0 = threadIdx.x; i0 < m * R; i0 += 8 * 256) {   // eight loads in flight, then the stores
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int idx = i0 + q * 256, c = idx / R, r = idx - c * R;
        v[q] = (idx < m * R && r < nr) ? A[(int64_t)c * nf + r0 + r] : (T)0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q * 256 < m * R) Xs[i0 + q * 256] = v[q];
    }
  const int rg = threadIdx.x % RG, cg = threadIdx.x / RG;
  // Global loads are issued ahead of their use, into registers: the inverse of the
  // next diagonal block during the current panel, the first 64-column chunk of L
  // below a panel before the panel's diagonal product, and each further chunk
  // while the previous one is applied.  A chunk exists only after a full 32-column
  // panel (jb == 32), so every chunk is 32 x 64 = 8 values per thread.
  // inv(L_jj), written by POTRF: column c at G[c * 32 .. c * 32 + 31]; L[l * 33 + c] = inv[c][l]
  const T* G0 = reinterpret_cast<const T*>(a.arenas.inv + (int64_t)s * a.arenas.inv_stride + nd.inv_off);
  constexpr int kInv = 1024 / 256, kPre = 32 * 64 / 256;
  T gin[kInv], pre[kPre];
#pragma unroll
  for (int k = 0; k < kInv; ++k) gin[k] = G0[threadIdx.x + k * 256];
  auto fetch = [&](int j0, int cn) {
#pragma unroll
    for (int k = 0; k < kPre; ++k) {
      const int idx = threadIdx.x + k * 256, l = idx >> 6, cc = idx & 63;
      pre[k] = (cn + cc < m) ? A[(int64_t)(j0 + l) * nf + cn + cc] : (T)0;
    }
  };
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int jb = min(32, m - j0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kInv; ++k) {
      const int idx = threadIdx.x + k * 256;
      L[(idx >> 5) * 33 + (idx & 31)] = gin[k];
    }
    __syncthreads();
    if (j0 + 32 < m)
#pragma unroll
      for (int k = 0; k < kInv; ++k) gin[k] = G0[(j0 / 32 + 1) * 1024 + threadIdx.x + k * 256];
    if (j0 + jb < m) fetch(j0, j0 + jb);
    // X_blk <- X_blk inv(L_jj)^T: x_c = sum_{l <= c} x_l inv[c][l]; each thread one row and a
    // group of columns, results kept in registers until all threads have read X_blk
    {
      constexpr int CPB = 32 * R / 256;        // columns per thread
      const int r = threadIdx.x % R, cbase = (threadIdx.x / R) * CPB;
      T acc[CPB];
#pragma unroll
      for (int q = 0; q < CPB; ++q) acc[q] = (T)0;
      for (int l = 0; l < jb; ++l) {
        const T x = X[(j0 + l) * ldx + r];
#pragma unroll
        for (int q = 0; q < CPB; ++q) {
          const int c = cbase + q;
          if (l <= c) acc[q] += x * L[l * 33 + c];
        }
      }
      __syncthreads();
      if (r < nr)
#pragma unroll
        for (int q = 0; q < CPB; ++q)
          if (cbase + q < jb) X[(j0 + cbase + q) * ldx + r] = acc[q];
    }
    // trailing chunks of 64 columns
    for (int c0 = j0 + jb; c0 < m; c0 += 64) {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kPre; ++k) Lc[threadIdx.x + k * 256] = pre[k];
      __syncthreads();
      if (c0 + 64 < m) fetch(j0, c0 + 64);
      T acc[4][CPT];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < CPT; ++w) acc[q][w] = (T)0;
      const int rr = rg * 4, cc0 = cg * CPT;
      for (int l = 0; l < jb; ++l) {
        const T* xc = X + (j0 + l) * ldx + rr;
        const T* lc = Lc + l * 64 + cc0;
        T x[4], y[CPT];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = xc[q];
#pragma unroll
        for (int w = 0; w < CPT; ++w) y[w] = lc[w];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < CPT; ++w) acc[q][w] += x[q] * y[w];
      }
#pragma unroll
      for (int w = 0; w < CPT; ++w) {
        const int c = c0 + cc0 + w;
        if (c < m) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (rr + q < nr) X[c * ldx + rr + q] -= acc[q][w];
        }
      }
    }
  }
  __syncthreads();
  if (in_smem)
    for (int idx = threadIdx.x; idx < m * R; idx += blockDim.x) {
      const int c = idx / R, rr = idx - c * R;
      if (rr < nr) A[(int64_t)c * nf + r0 + rr] = Xs[idx];
    }
  if (r0 + nr == nf) {   // this block holds the bordered row: y_g
    T* Y = node_Y<T>(a.arenas, nd, s);
    for (int c = threadIdx.x; c < m; c += blockDim.x) Y[c] = X[c * ldx + (nr - 1)];
  }
  if (std::is_same<T, float>::value && nd.tc_off >= 0)
    write_tc_tiles(reinterpret_cast<const float*>(X), ldx, nd, a.arenas, s, blockIdx.x * R, nr, r0 + nr == nf);
}

// TRSM of the large FP32 fronts, X = K_Bg L_gg^-T over the rows below gamma (the
// bordered row included), the same blocked arithmetic as k_trsm with wider trailing
// updates: 32 rows per CTA with their m columns in shared memory; per 32-column panel
// X_p <- X_p inv(L_pp)^T (the inverted diagonal block that POTRF wrote), then the
// columns to its right in 128-column chunks, X_c -= X_p L_cp^T, each thread a 4 x 4
// register tile (two 16-byte shared loads per 16 multiply-adds; the 4 x 2 tile of
// k_trsm spent six scalar loads per eight).  The next chunk of L (32 x 128, 16 values
// per thread) is loaded into registers while the current one is applied, the next
// inverted block during the panel.
constexpr int kTrwR = 32, kTrwC = 128, kTrwCap = 760;

__global__ void __launch_bounds__(256, 3) k_trsm_wide(StepArgs a) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m;
  const int r0 = m + blockIdx.x * kTrwR;
  if (r0 >= nf || m == 0) return;
  const int nr = min(kTrwR, nf - r0);
  float* A = node_F<float>(a.arenas, nd, s);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* L = reinterpret_cast<float*>(smem_raw);   // [32][36]: L[l][c] = inv(L_pp)[c][l]
  float* Lc = L + 32 * 36;                         // [32][kTrwC] the panel's columns right of it
  float* X = Lc + 32 * kTrwC;                      // [m][32] the CTA's rows
  const int tid = threadIdx.x;
  for (int i0 = tid; i0 < m * kTrwR; i0 += 8 * 256) {   // eight loads in flight, then the stores
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int idx = i0 + q * 256, c = idx >> 5, r = idx & 31;
      v[q] = (idx < m * kTrwR && r < nr) ? A[(int64_t)c * nf + r0 + r] : 0.0f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (i0 + q * 256 < m * kTrwR) X[i0 + q * 256] = v[q];
  }
  const float* G0 = reinterpret_cast<const float*>(a.arenas.inv + (int64_t)s * a.arenas.inv_stride + nd.inv_off);
  float gin[4], pre[16];
#pragma unroll
  for (int k = 0; k < 4; ++k) gin[k] = G0[tid + k * 256];
  // chunk (j0, c0): Lc[l][cc] = L[c0 + cc][j0 + l] = A[(j0 + l) nf + c0 + cc]; thread t
  // loads column cc = t & 127 of rows l = 2 k + (t >> 7)
  const int fc = tid & (kTrwC - 1), fl = tid >> 7;
  auto fetch = [&](int j0, int c0) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
      pre[k] = (c0 + fc < m) ? A[(int64_t)(j0 + 2 * k + fl) * nf + c0 + fc] : 0.0f;
  };
  const int rg = tid & 7, cg = tid >> 3;   // update tile: rows 4 rg .. 4 rg + 3, columns 4 cg .. 4 cg + 3
  for (int j0 = 0; j0 < m; j0 += 32) {
    const int jb = min(32, m - j0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {   // G0[l * 32 + c] = inv[c][l] -> L[l][c], zero where c < l
      const int idx = tid + k * 256, l = idx >> 5, c = idx & 31;
      L[l * 36 + c] = l <= c ? gin[k] : 0.0f;
    }
    __syncthreads();
    if (j0 + 32 < m)
#pragma unroll
      for (int k = 0; k < 4; ++k) gin[k] = G0[(j0 / 32 + 1) * 1024 + tid + k * 256];
    if (j0 + jb < m) fetch(j0, j0 + jb);   // a full panel (jb = 32) precedes any chunk
    {   // X_p <- X_p inv(L_pp)^T: x_c = sum_{l <= c} x_l inv[c][l]; one row, four columns per
        // thread, over l <= the last of them only (the inverse is lower triangular)
      const int r = tid & 31, cb = (tid >> 5) * 4;
      float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      const int lend = min(jb, cb + 4);
      for (int l = 0; l < lend; ++l) {
        const float x = X[(j0 + l) * kTrwR + r];
        const float4 g = *reinterpret_cast<const float4*>(L + l * 36 + cb);
        acc[0] += x * g.x;
        acc[1] += x * g.y;
        acc[2] += x * g.z;
        acc[3] += x * g.w;
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (cb + q < jb) X[(j0 + cb + q) * kTrwR + r] = acc[q];
    }
    for (int c0 = j0 + jb; c0 < m; c0 += kTrwC) {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 16; ++k) Lc[(2 * k + fl) * kTrwC + fc] = pre[k];
      __syncthreads();
      if (c0 + kTrwC < m) fetch(j0, c0 + kTrwC);
      if (c0 + 4 * cg >= m) continue;   // no column of this thread's tile in the chunk
      float acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = 0.0f;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        const float4 x = *reinterpret_cast<const float4*>(X + (j0 + l) * kTrwR + 4 * rg);
        const float4 y = *reinterpret_cast<const float4*>(Lc + l * kTrwC + 4 * cg);
        const float xv[4] = {x.x, x.y, x.z, x.w};
        const float yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] += xv[q] * yv[w];
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int c = c0 + 4 * cg + w;
        if (c < m) {
          float4* xc = reinterpret_cast<float4*>(X + c * kTrwR + 4 * rg);
          float4 v = *xc;
          v.x -= acc[0][w]; v.y -= acc[1][w]; v.z -= acc[2][w]; v.w -= acc[3][w];
          *xc = v;
        }
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * kTrwR; idx += blockDim.x) {
    const int c = idx >> 5, r = idx & 31;
    if (r < nr) A[(int64_t)c * nf + r0 + r] = X[idx];
  }
  if (r0 + nr == nf) {   // this block holds the bordered row: y_g
    float* Y = node_Y<float>(a.arenas, nd, s);
    for (int c = tid; c < m; c += blockDim.x) Y[c] = X[c * kTrwR + (nr - 1)];
  }
  if (nd.tc_off >= 0) write_tc_tiles(X, kTrwR, nd, a.arenas, s, blockIdx.x * kTrwR, nr, r0 + nr == nf);
}

// SYRK: S -= X X^T with X = F[m:nf, 0:m] (b+1 rows incl. the right-hand side).
// One CTA per (64 x 64 lower tile pair, node, sample), 4 x 4 per thread.
constexpr int kSyrkTile = 64, kSyrkK = 16;

template <typename T>
__global__ void k_syrk(StepArgs a) {
  const int node = a.list[blockIdx.y];
  const int s = blockIdx.z;
  bind_plan(a, node);
  if (s >= a.batch) return;
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
  T sv[4][4];   // loads first (in flight together), then the stores
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = TI * kSyrkTile + ty + 16 * q;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int j = TJ * kSyrkTile + tx + 16 * w;
      sv[q][w] = (i < nb && j < nb && i >= j) ? S[(int64_t)j * nb + i] : (T)0;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = TI * kSyrkTile + ty + 16 * q;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int j = TJ * kSyrkTile + tx + 16 * w;
      if (i < nb && j < nb && i >= j) S[(int64_t)j * nb + i] = sv[q][w] - acc[q][w];
    }
  }
}

// The bordered right-hand-side row of S for fronts whose SYRK runs on the tensor
// cores: S[b, j] = (sons' entries at (rhs, m + j)) - sum_k y_k X[j, k] for
// j = 0..b (y = the last row of X), one CTA per (node, sample), threads over j
// (coalesced down the columns of F).  The sons' entries are gathered here: the
// fill of these fronts writes only the gamma columns.
__global__ void k_syrk_rhs(StepArgs a) {
  const int node = a.list[blockIdx.x];
  const int s = blockIdx.y;
  bind_plan(a, node);
  if (s >= a.batch) return;
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m, b = nd.b, nb = b + 1;
  if (m == 0) return;
  const float* X = a.arenas.f32 + (int64_t)s * a.arenas.f32_stride + nd.f_off + m;
  float* S = a.arenas.s32 + (int64_t)s * a.arenas.s32_stride + nd.s_off;
  const int32_t* map = a.maps + nd.map_off;
  const NodeDev c0 = nd.leaf ? nd : a.nodes[nd.child0], c1 = nd.leaf ? nd : a.nodes[nd.child1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* y = reinterpret_cast<float*>(smem_raw);
  for (int k = threadIdx.x; k < m; k += blockDim.x) y[k] = X[(int64_t)k * nf + b];
  __syncthreads();
  for (int j = threadIdx.x; j <= b; j += blockDim.x) {
    float acc = 0.0f;
    int k = 0;
    for (; k + 16 <= m; k += 16) {   // sixteen column loads in flight, then the products
      float x[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) x[q] = X[(int64_t)(k + q) * nf + j];
#pragma unroll
      for (int q = 0; q < 16; ++q) acc += y[k + q] * x[q];
    }
    for (; k < m; ++k) acc += y[k] * X[(int64_t)k * nf + j];
    const float g = nd.leaf ? S[(int64_t)j * nb + b]
                            : father_entry<float>(nf - 1, m + j, s, nd, map, c0, c1, a.arenas, a.rhs);
    S[(int64_t)j * nb + b] = g - acc;
  }
}

template <typename T>
cudaError_t launch_front_large(const StepArgs& a, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  {
    // FP32 fronts: the tensor-core Schur update gathers the sons' boundary block
    // itself, so only the gamma columns are filled
    const bool gamma_only = std::is_same<T, float>::value;
    const int cols = (gamma_only && a.max_rect == 0) ? a.max_m : a.max_nf;   // max_rect > 0: the list has leaves
    dim3 grid((cols + 7) / 8, a.nlist, a.batch);
    if (a.prof) a.prof->begin(kProfFill, 0.0, st);
    k_front_fill<T><<<grid, 256, 0, st>>>(a, gamma_only ? 1 : 0);
    if (a.prof) a.prof->end(st);
  }
  const size_t rows_smem = (size_t)min(a.max_m, SmemCap<T>::rows);
  const bool fused_pt = a.max_m <= 32 || (sizeof(T) == 4 && a.max_m <= 64);
  if (fused_pt) {   // POTRF and TRSM in one kernel (two 32-column blocks in FP32 only: registers)
    if (a.prof) a.prof->begin(kProfCholTrsm, a.fl_chol + a.fl_trsm, st);
    const dim3 grid(a.nlist, (a.batch + kCholTrsmWarps - 1) / kCholTrsmWarps);
    if (a.max_m <= 32)
      k_chol_trsm<T, 1><<<grid, 32 * kCholTrsmWarps, kCholTrsmWarps * sizeof(CholTrsmSmem<T, 1>), st>>>(a);
    else
      k_chol_trsm<T, 2><<<grid, 32 * kCholTrsmWarps, kCholTrsmWarps * sizeof(CholTrsmSmem<T, 2>), st>>>(a);
    if (a.prof) a.prof->end(st);
  } else {
    size_t tri_bytes = 0;
    if (a.prof) a.prof->begin(kProfPotrf, a.fl_chol, st);
    if (potrf_in_smem<T>(a.max_m, &tri_bytes)) {
      k_potrf_smem<T><<<dim3(a.nlist, a.batch), 256, tri_bytes, st>>>(a);
    } else {
      const size_t smem = (((rows_smem + 3) & ~(size_t)3) * kPanel + 2 * 32 * kWs + 32) * sizeof(T);
      k_potrf<T><<<dim3(a.nlist, a.batch), 256, smem, st>>>(a);
    }
    if (a.prof) a.prof->end(st);
  }
  if (!fused_pt && std::is_same<T, float>::value && a.max_m <= kTrwCap) {
    const size_t smem = ((size_t)a.max_m * kTrwR + 32 * 36 + 32 * kTrwC) * sizeof(float);
    dim3 grid((a.max_b + 1 + kTrwR - 1) / kTrwR, a.nlist, a.batch);
    if (a.prof) a.prof->begin(kProfTrsm, a.fl_trsm, st);
    k_trsm_wide<<<grid, 256, smem, st>>>(a);
    if (a.prof) a.prof->end(st);
  } else if (!fused_pt) {
    constexpr int R = TrsmShape<T>::rows;
    const size_t xrows = (size_t)min(a.max_m, TrsmShape<T>::cap);
    const size_t smem = (xrows * R + 32 * 33 + 3 + 32 * 64) * sizeof(T) + 16;
    dim3 grid((a.max_b + 1 + R - 1) / R, a.nlist, a.batch);
    if (a.prof) a.prof->begin(kProfTrsm, a.fl_trsm, st);
    k_trsm<T, 32><<<grid, 256, smem, st>>>(a);
    if (a.prof) a.prof->end(st);
  }
  if (std::is_same<T, float>::value) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.prof) a.prof->begin(kProfSyrkTc, a.fl_syrk, st);
    e = launch_syrk_tc(a, st);   // tensor cores, 3xTF32, boundary rows
    if (a.prof) a.prof->end(st);
    if (e != cudaSuccess) return e;
    if (a.prof) a.prof->begin(kProfSyrkRhs, a.fl_rhs, st);
    k_syrk_rhs<<<dim3(a.nlist, a.batch), 256, (size_t)a.max_m * sizeof(float), st>>>(a);
    if (a.prof) a.prof->end(st);
    return cudaGetLastError();
  }
  {
    const int nt = (a.max_b + 1 + kSyrkTile - 1) / kSyrkTile;
    dim3 grid(nt * (nt + 1) / 2, a.nlist, a.batch);
    if (a.prof) a.prof->begin(kProfSyrk, a.fl_syrk + a.fl_rhs, st);
    k_syrk<T><<<grid, 256, 0, st>>>(a);
    if (a.prof) a.prof->end(st);
  }
  return cudaGetLastError();
}

template cudaError_t launch_front_large<double>(const StepArgs&, cudaStream_t);
template cudaError_t launch_front_large<float>(const StepArgs&, cudaStream_t);

cudaError_t configure_front_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_potrf<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf_smem<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf_smem<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_trsm<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_trsm<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_chol_trsm<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm<float, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_trsm_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
