// Device helpers shared by the HDD kernels: front entries (leaf assembly and
// father-system extend-add), status codes, small math.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "plan.h"

namespace hdd {

// Per-sample failure code: (-status) | (node << 8), first failure wins.
__device__ __forceinline__ void flag_status(int32_t* status, int s, int code, int node) {
  if (status) atomicCAS(status + s, 0, code | (node << 8));
}

// Right-hand-side entry of vertex v for sample s: the load h^2 f of vertex
// quadrature (Sec. 3.1, Eq. coefc with |t|/3 per triangle, six triangles per
// vertex) or a caller vector (residual of iterative refinement).
struct Rhs {
  const double* vec;   // [batch x N^2] or nullptr
  int64_t stride;
  double constant;
  __device__ __forceinline__ double operator()(int s, int v) const {
    return vec ? vec[(int64_t)s * stride + v] : constant;
  }
};

// kappa of triangle (cell (i, j), half t) if the cell lies in the rectangle.
template <typename KT>
__device__ __forceinline__ KT kap_in(const KT* kap, int N, const NodeDev& nd, int i, int j, int t) {
  if (i < nd.x0 || i >= nd.x1 || j < nd.y0 || j >= nd.y1) return (KT)0;
  return kap[2 * ((int64_t)j * (N - 1) + i) + t];
}
// Stiffness weight of an axis edge from the triangles inside the rectangle.  For
// the right isosceles triangles of this mesh the P1 element matrix (Eq. coefA)
// is kappa_t * [[1/2, -1/2, 0], [-1/2, 1, -1/2], [0, -1/2, 1/2]] (right-angle
// vertex in the middle): each leg couples its ends by -kappa_t/2, the hypotenuse
// by 0.  The horizontal edge (i,j)-(i+1,j) is a leg of the lower-right triangle
// of cell (i,j) and of the upper-left triangle of cell (i,j-1).
template <typename KT>
__device__ __forceinline__ KT w_horizontal(const KT* kap, int N, const NodeDev& nd, int i, int j) {
  return (KT)0.5 * (kap_in(kap, N, nd, i, j, 0) + kap_in(kap, N, nd, i, j - 1, 1));
}
// The vertical edge (i,j)-(i,j+1) is a leg of the upper-left triangle of cell
// (i,j) and of the lower-right triangle of cell (i-1,j).
template <typename KT>
__device__ __forceinline__ KT w_vertical(const KT* kap, int N, const NodeDev& nd, int i, int j) {
  return (KT)0.5 * (kap_in(kap, N, nd, i, j, 1) + kap_in(kap, N, nd, i - 1, j, 0));
}

// Entry (r, c), r >= c, of a leaf front: the stiffness of the leaf's own
// triangles over [interior, boundary, rhs] (Leaves to Root, step 1).  The load
// enters at the interior rows only; boundary rows receive theirs at the node
// that eliminates them.  Computed in the front's precision KT.
template <typename KT>
__device__ __forceinline__ KT leaf_entry(int r, int c, int s, const NodeDev& nd, const int32_t* vid,
                                         const KT* kap, int N, const Rhs& rhs) {
  const int nf = nd.nf;
  if (r == nf - 1) return (c < nd.m) ? (KT)rhs(s, vid[c]) : (KT)0;
  const int v = vid[r], u = vid[c];
  const int vi = v % N, vj = v / N;
  if (v == u) {
    return w_horizontal(kap, N, nd, vi - 1, vj) + w_horizontal(kap, N, nd, vi, vj) +
           w_vertical(kap, N, nd, vi, vj - 1) + w_vertical(kap, N, nd, vi, vj);
  }
  const int ui = u % N, uj = u / N;
  if (vj == uj && (vi - ui == 1 || ui - vi == 1)) return -w_horizontal(kap, N, nd, min(vi, ui), vj);
  if (vi == ui && (vj - uj == 1 || uj - vj == 1)) return -w_vertical(kap, N, nd, vi, min(vj, uj));
  return (KT)0;
}

// Workspace arenas of one precision pair (per-sample strides in elements).
struct Arenas {
  double* f64; int64_t f64_stride;
  float* f32; int64_t f32_stride;
  double* s64; int64_t s64_stride;
  float* s32; int64_t s32_stride;
  double* y64; int64_t y64_stride;
  float* y32; int64_t y32_stride;
  unsigned char* tc; int64_t tc_stride;   // split TF32 tiles for the tensor-core SYRK
  unsigned char* inv; int64_t inv_stride; // inverted diagonal blocks of L_gg (POTRF -> TRSM)
};

// y_g of a node (the bordered row of its front): written by the upsweep and by
// every right-hand-side sweep, read by the descent.
template <typename T> __device__ __forceinline__ T* node_Y(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* node_Y<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.y64 + (int64_t)s * A.y64_stride + nd.y_off;
}
template <> __device__ __forceinline__ float* node_Y<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.y32 + (int64_t)s * A.y32_stride + nd.y_off;
}

// Entry (a, b) of a son's Schur complement (lower triangle is stored), returned
// in the caller's precision T; the son's own precision is read directly.
template <typename T>
__device__ __forceinline__ T son_entry(const Arenas& A, const NodeDev& ch, int s, int a, int b) {
  const int lo = min(a, b), hi = max(a, b);
  const int64_t idx = (int64_t)lo * (ch.b + 1) + hi + ch.s_off;
  return ch.fp64 ? (T)A.s64[(int64_t)s * A.s64_stride + idx] : (T)A.s32[(int64_t)s * A.s32_stride + idx];
}

// Entry (r, c), r >= c, of a father front (Sec. 3.3, Eq. block_equation4): the
// sons' Schur complements embedded into the union of their boundaries and added
// (the shared interface block receives both), plus the load of the father's own
// gamma vertices in the right-hand-side row.
template <typename T>
__device__ __forceinline__ T father_entry(int r, int c, int s, const NodeDev& nd, const int32_t* map,
                                          const NodeDev& ch0, const NodeDev& ch1, const Arenas& A,
                                          const Rhs& rhs) {
  const int nf = nd.nf;
  const int32_t* pos0 = map + (nf - 1);
  const int32_t* pos1 = pos0 + nf;
  T v = (T)0;
  int a = pos0[r], b = pos0[c];
  if (a >= 0 && b >= 0) v += son_entry<T>(A, ch0, s, a, b);
  a = pos1[r]; b = pos1[c];
  if (a >= 0 && b >= 0) v += son_entry<T>(A, ch1, s, a, b);
  if (r == nf - 1 && c < nd.m) v += (T)rhs(s, map[c]);
  return v;
}

// kappa per triangle in the front's precision (FP64 array, or its FP32 copy).
template <typename T> __device__ __forceinline__ const T* kappa_of(const double* k64, const float* k32);
template <> __device__ __forceinline__ const double* kappa_of<double>(const double* k64, const float*) { return k64; }
template <> __device__ __forceinline__ const float* kappa_of<float>(const double*, const float* k32) { return k32; }

template <typename T> struct Prec;
template <> struct Prec<double> { static constexpr bool is64 = true; };
template <> struct Prec<float> { static constexpr bool is64 = false; };

}  // namespace hdd
