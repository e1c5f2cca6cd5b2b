// Mean values of the solution over every subdomain of the tree (Sec. 5, Eq. mean;
// Sec. 5.1).  For a piecewise linear u the integral over a triangle t is
// |t|/3 (u_1 + u_2 + u_3); a leaf's mean is the sum over its triangles divided by
// its area.  A father's mean follows from its sons' as in Sec. 5.1: the functional
// of omega is c_1 times that of omega_1 plus c_2 times that of omega_2, with
// c_i = |omega_i| / |omega| (the sons' rectangles tile the father's and meet on the
// interface, which has no area).
#include "launch.h"

namespace hdd {

// One thread per (leaf, sample).  Cell (i, j) holds the lower-right triangle
// (i,j), (i+1,j), (i+1,j+1) and the upper-left one (i,j), (i+1,j+1), (i,j+1),
// each of area h^2 / 2, so the cell adds h^2 / 6 times (2 u(i,j) + u(i+1,j) +
// 2 u(i+1,j+1) + u(i,j+1)).  Summed over the leaf's cells every vertex enters
// once with the sum of those corner weights over the cells it belongs to (6 at an
// inner vertex); the leaf's area is cells * h^2, so h^2 cancels.
__global__ void k_leaf_means(const NodeDev* __restrict__ nodes, const int32_t* __restrict__ list, int n,
                             const double* __restrict__ u, int64_t u_stride, int N, double* __restrict__ means,
                             int64_t m_stride) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (q >= n) return;
  const int node = list[q];
  const NodeDev nd = nodes[node];
  const double* us = u + (int64_t)s * u_stride;
  double acc = 0.0;
  for (int j = nd.y0; j <= nd.y1; ++j) {
    const double* row = us + (int64_t)j * N;
    const bool up = j < nd.y1, down = j > nd.y0;   // cells above / below this vertex row
    for (int i = nd.x0; i <= nd.x1; ++i) {
      const bool right = i < nd.x1, left = i > nd.x0;
      // corner (i,j) of cell (i,j): 2; of cell (i-1,j): 1; of cell (i-1,j-1): 2; of cell (i,j-1): 1
      const int wgt = (up ? (right ? 2 : 0) + (left ? 1 : 0) : 0) + (down ? (left ? 2 : 0) + (right ? 1 : 0) : 0);
      acc += (double)wgt * row[i];
    }
  }
  const double cells = (double)(nd.x1 - nd.x0) * (double)(nd.y1 - nd.y0);
  means[(int64_t)s * m_stride + node] = acc / (6.0 * cells);
}

// One thread per (father, sample) of one height: mean = c_1 mean_1 + c_2 mean_2.
__global__ void k_father_means(const NodeDev* __restrict__ nodes, const int32_t* __restrict__ list, int n,
                               double* __restrict__ means, int64_t m_stride) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (q >= n) return;
  const int node = list[q];
  const NodeDev nd = nodes[node];
  const NodeDev s0 = nodes[nd.child0], s1 = nodes[nd.child1];
  auto area = [](const NodeDev& x) { return (double)(x.x1 - x.x0) * (double)(x.y1 - x.y0); };
  const double a = area(nd);
  double* ms = means + (int64_t)s * m_stride;
  ms[node] = (area(s0) / a) * ms[nd.child0] + (area(s1) / a) * ms[nd.child1];
}

cudaError_t launch_leaf_means(const NodeDev* nodes, const int32_t* list, int n, const double* u, int64_t u_stride,
                              int N, double* means, int64_t m_stride, int batch, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_leaf_means<<<dim3((n + 127) / 128, batch), 128, 0, st>>>(nodes, list, n, u, u_stride, N, means, m_stride);
  return cudaGetLastError();
}

cudaError_t launch_father_means(const NodeDev* nodes, const int32_t* list, int n, double* means, int64_t m_stride,
                                int batch, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_father_means<<<dim3((n + 127) / 128, batch), 128, 0, st>>>(nodes, list, n, means, m_stride);
  return cudaGetLastError();
}

}  // namespace hdd
