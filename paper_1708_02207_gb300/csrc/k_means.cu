// Mean values of the solution over every subdomain of the tree (Sec. 5, Eq. mean;
// Sec. 5.1).  For a piecewise linear u the integral over a triangle t is
// |t|/3 (u_1 + u_2 + u_3); a leaf's mean is the sum over its triangles divided by
// its area.  A father's mean follows from its sons' as in Sec. 5.1: the functional
// of omega is c_1 times that of omega_1 plus c_2 times that of omega_2, with
// c_i = |omega_i| / |omega| (the sons' rectangles tile the father's and meet on the
// interface, which has no area).
#include "launch.h"

namespace hdd {

// One warp per (leaf, sample), lanes over the leaf's cells (row by row, so that
// the lanes of one cell row read consecutive vertices).  Cell (i, j) holds the
// lower-right triangle (i,j), (i+1,j), (i+1,j+1) and the upper-left one (i,j),
// (i+1,j+1), (i,j+1), each of area h^2 / 2: the cell adds h^2 / 6 times the two
// corner sums, and the leaf's area is cells * h^2, so h^2 cancels.  The lane sums
// are combined by a fixed butterfly, so the result does not depend on timing.
constexpr int kMeanWarps = 8;
__global__ void __launch_bounds__(32 * kMeanWarps) k_leaf_means(const NodeDev* __restrict__ nodes,
                                                                const int32_t* __restrict__ list, int n,
                                                                const double* __restrict__ u, int64_t u_stride,
                                                                int N, double* __restrict__ means,
                                                                int64_t m_stride) {
  const int q = blockIdx.x * kMeanWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.y;
  if (q >= n) return;   // uniform per warp
  const int node = list[q];
  const NodeDev nd = nodes[node];
  const double* us = u + (int64_t)s * u_stride;
  const int w = nd.x1 - nd.x0, cells = w * (nd.y1 - nd.y0);
  double acc = 0.0;
  for (int c = lane; c < cells; c += 32) {
    const int i = nd.x0 + c % w, j = nd.y0 + c / w;
    const double* lo = us + (int64_t)j * N + i;
    const double* hi = lo + N;
    const double a = lo[0], b = lo[1], cc = hi[1], d = hi[0];
    acc += (a + b + cc) + (a + cc + d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) means[(int64_t)s * m_stride + node] = acc / (6.0 * (double)cells);
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
  k_leaf_means<<<dim3((n + kMeanWarps - 1) / kMeanWarps, batch), 32 * kMeanWarps, 0, st>>>(nodes, list, n, u,
                                                                                          u_stride, N, means,
                                                                                          m_stride);
  return cudaGetLastError();
}

cudaError_t launch_father_means(const NodeDev* nodes, const int32_t* list, int n, double* means, int64_t m_stride,
                                int batch, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_father_means<<<dim3((n + 127) / 128, batch), 128, 0, st>>>(nodes, list, n, means, m_stride);
  return cudaGetLastError();
}

}  // namespace hdd
