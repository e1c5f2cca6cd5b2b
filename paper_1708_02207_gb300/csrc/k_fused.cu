// Fused bottom of the upsweep ("Leaves to Root", Sec. 3.4): one CTA of 16 warps
// eliminates a whole subtree of the decomposition tree for one sample, level by
// level, keeping every Schur complement of the subtree (Psi_omega, Sec. 2.4) in
// shared memory.  Only the factors of every node (needed by the descent and by
// the refinement sweeps) and the Schur complement of the subtree's root go to
// global memory.  Nodes of one level are shared out among warp groups:
//   * fronts of at most 32 rows handled by a single warp: one row per lane in
//     registers, Cholesky with shuffles;
//   * otherwise a group of warps per front in shared memory with a blocked
//     right-looking partial Cholesky, synchronised by a named barrier per group.
// Schur blocks inside the subtree are stored as full symmetric squares.
#include "launch.h"

namespace hdd {

namespace {

constexpr unsigned kAll = 0xffffffffu;
constexpr int kFuseWarps = 16;

__device__ __forceinline__ void group_sync(int id, int nthreads) {
  if (nthreads == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
  }
}

template <typename T> __device__ __forceinline__ T* fF(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* fF<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* fF<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* fS(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* fS<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* fS<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

__host__ __device__ __forceinline__ int fuse_ld(int nf) {
  int ld = (nf + 3) & ~3;
  if ((ld & 7) == 0) ld += 4;
  return ld;
}

// ---------------------------------------------------------------------------
// One warp, front of at most 32 rows (lane r = row r).  Sons' Schur complements
// come from shared memory (full squares at son_off).  Output: factor columns
// and y_g to global memory; the Schur block as a full square either into shared
// memory (Ssm) or, for the subtree root, into the global Schur arena (lower).
template <typename T>
__device__ void warp_front(const FuseArgs& f, int node, const NodeDev& nd, int s, const T* Sprev, T* Ssm) {
  const StepArgs& a = f.a;
  const int lane = threadIdx.x & 31;
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1, N = a.N;
  const int32_t* map = a.maps + nd.map_off;
  const int v = (lane < nf - 1) ? map[lane] : -1;
  const T rv = (lane < m) ? (T)a.rhs(s, v) : (T)0;
  T row[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) row[c] = (T)0;
  if (nd.leaf) {
    const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)s * a.kap_stride;
    int vi = -7, vj = -7;
    T wl = (T)0, wr = (T)0, wd = (T)0, wu = (T)0;
    if (v >= 0) {
      vi = v % N;
      vj = v / N;
      wl = w_horizontal(kap, N, nd, vi - 1, vj);
      wr = w_horizontal(kap, N, nd, vi, vj);
      wd = w_vertical(kap, N, nd, vi, vj - 1);
      wu = w_vertical(kap, N, nd, vi, vj);
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int ci = __shfl_sync(kAll, vi, c), cj = __shfl_sync(kAll, vj, c);
      const T rc = __shfl_sync(kAll, rv, c);
      T val = (T)0;
      if (c < nf && lane < nf) {
        if (lane == nf - 1) val = (c < m) ? rc : (T)0;
        else if (c == nf - 1) val = rv;
        else if (c == lane) val = wl + wr + wd + wu;
        else if (cj == vj && ci == vi - 1) val = -wl;
        else if (cj == vj && ci == vi + 1) val = -wr;
        else if (ci == vi && cj == vj - 1) val = -wd;
        else if (ci == vi && cj == vj + 1) val = -wu;
      }
      row[c] = val;
    }
  } else {
    const int32_t* pos0 = map + (nf - 1);
    const int32_t* pos1 = pos0 + nf;
    const NodeDev c0 = a.nodes[nd.child0], c1 = a.nodes[nd.child1];
    const T* S0 = Sprev + f.fuse_soff[nd.child0];
    const T* S1 = Sprev + f.fuse_soff[nd.child1];
    const int ld0 = c0.b + 1, ld1 = c1.b + 1;
    const int p0 = (lane < nf) ? pos0[lane] : -1, p1 = (lane < nf) ? pos1[lane] : -1;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int q0 = __shfl_sync(kAll, p0, c), q1 = __shfl_sync(kAll, p1, c);
      const T rc = __shfl_sync(kAll, rv, c);
      T val = (T)0;
      if (p0 >= 0 && q0 >= 0) val += S0[p0 * ld0 + q0];
      if (p1 >= 0 && q1 >= 0) val += S1[p1 * ld1 + q1];
      if (lane == nf - 1 && c < m) val += rc;
      if (c == nf - 1 && lane < m) val += rv;
      row[c] = val;
    }
  }
  bool bad = false;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < m) {
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
  if (bad && lane == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
  T* F = fF<T>(a.arenas, nd, s);
#pragma unroll
  for (int c = 0; c < 32; ++c)
    if (c < m && lane < nf) F[c * nf + lane] = row[c];
  if (lane == nf - 1) {
    T* Y = node_Y<T>(a.arenas, nd, s);
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c < m) Y[c] = row[c];
  }
  if (Ssm) {
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c >= m && c < nf && lane >= m && lane < nf) Ssm[(c - m) * nb + (lane - m)] = row[c];
  } else {
    T* S = fS<T>(a.arenas, nd, s);
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c >= m && c < nf && lane >= c && lane < nf) S[(c - m) * nb + (lane - m)] = row[c];
  }
}

// ---------------------------------------------------------------------------
// A group of warps (gt threads, group-local thread id t, barrier id bid), front
// in shared memory K (column-major, ld fuse_ld(nf)).
template <typename T>
__device__ void group_front(const FuseArgs& f, int node, const NodeDev& nd, int s, const T* Sprev, T* Ssm, T* K,
                            int t, int gt, int bid) {
  const StepArgs& a = f.a;
  const int nf = nd.nf, m = nd.m, ld = fuse_ld(nf), nb = nd.b + 1;
  const int warp = t >> 5, lane = t & 31, nwarp = gt >> 5;
  const int32_t* map = a.maps + nd.map_off;
  if (nd.leaf) {
    const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)s * a.kap_stride;
    for (int c = warp; c < nf; c += nwarp)
      for (int r = lane; r < nf; r += 32) K[c * ld + r] = (r >= c) ? leaf_entry<T>(r, c, s, nd, map, kap, a.N, a.rhs) : (T)0;
  } else {
    for (int idx = t; idx < nf * ld; idx += gt) K[idx] = (T)0;
    group_sync(bid, gt);
    for (int sc = 0; sc < 2; ++sc) {
      const int cn = sc ? nd.child1 : nd.child0;
      const NodeDev ch = a.nodes[cn];
      const T* Sc = Sprev + f.fuse_soff[cn];
      const int ldc = ch.b + 1;
      const int32_t* up = a.maps + ch.up_off;
      for (int cc = warp; cc < ldc; cc += nwarp) {
        const int pc = up[cc];
        for (int aa = cc + lane; aa < ldc; aa += 32) {
          const int pr = up[aa];
          K[min(pr, pc) * ld + max(pr, pc)] += Sc[cc * ldc + aa];
        }
      }
      group_sync(bid, gt);
    }
    for (int c = t; c < m; c += gt) K[c * ld + nf - 1] += (T)a.rhs(s, map[c]);
  }
  constexpr int kPB = 8;
  for (int k0 = 0; k0 < m; k0 += kPB) {
    const int kb = min(kPB, m - k0), kend = k0 + kb;
    for (int k = k0; k < kend; ++k) {
      group_sync(bid, gt);
      T p = K[k * ld + k];
      if (!(p > (T)0) || !isfinite(p)) {
        if (t == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);
        p = (T)1;
      }
      const T d = sqrt(p), inv = (T)1 / d;
      T* colk = K + k * ld;
      for (int i = k + 1 + t; i < nf; i += gt) colk[i] *= inv;
      group_sync(bid, gt);
      if (t == 0) colk[k] = d;
      for (int j = k + 1 + warp; j < kend; j += nwarp) {
        const T lj = colk[j];
        T* colj = K + j * ld;
        for (int i = j + lane; i < nf; i += 32) colj[i] -= colk[i] * lj;
      }
    }
    group_sync(bid, gt);
    if (kend >= nf) continue;
    const int t0 = kend & ~3;
    const int nt = (nf - t0 + 3) >> 2;
    for (int tj = warp; tj < nt; tj += nwarp) {
      const int j0 = t0 + 4 * tj;
      for (int ti = tj + lane; ti < nt; ti += 32) {
        const int i0 = t0 + 4 * ti;
        T acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
        for (int l = k0; l < kend; ++l) {
          const T* col = K + l * ld;
          T x[4], y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            x[q] = col[i0 + q];
            y[q] = col[j0 + q];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int j = j0 + w;
          if (j < kend || j >= nf) continue;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int i = i0 + q;
            if (i < nf && i >= j) K[j * ld + i] -= acc[q][w];
          }
        }
      }
    }
  }
  group_sync(bid, gt);
  T* F = fF<T>(a.arenas, nd, s);
  for (int c = warp; c < m; c += nwarp)
    for (int r = lane; r < nf; r += 32) F[c * nf + r] = K[c * ld + r];
  T* Y = node_Y<T>(a.arenas, nd, s);
  for (int c = t; c < m; c += gt) Y[c] = K[c * ld + nf - 1];
  if (Ssm) {
    for (int c = warp; c < nb; c += nwarp)
      for (int r = c + lane; r < nb; r += 32) {
        const T v = K[(m + c) * ld + m + r];
        Ssm[c * nb + r] = v;
        Ssm[r * nb + c] = v;
      }
  } else {
    T* S = fS<T>(a.arenas, nd, s);
    for (int c = warp; c < nb; c += nwarp)
      for (int r = c + lane; r < nb; r += 32) S[c * nb + r] = K[(m + c) * ld + m + r];
  }
}

}  // namespace

// One CTA per (fusion subtree, sample).  Subtree descriptor (12 ints per root):
// [0] offset of its node list (bottom-up, by height), [1] number of levels L,
// [2 .. 2+L] start of each level in the list.
template <typename T>
__global__ void __launch_bounds__(kFuseWarps * 32) k_subtree(FuseArgs f) {
  const int r = blockIdx.x, s = blockIdx.y;
  const int32_t* d = f.roots + r * 12;
  const int32_t* list = f.fused + d[0];
  const int L = d[1];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Sbuf0 = reinterpret_cast<T*>(smem_raw);
  T* Sbuf1 = Sbuf0 + f.sbuf_elems;
  T* Fw = Sbuf1 + f.sbuf_elems;
  const int warp = threadIdx.x >> 5;
  for (int h = 0; h < L; ++h) {
    const int beg = d[2 + h], end = d[3 + h], nh = end - beg;
    int wpf = kFuseWarps / nh;
    if (wpf < 1) wpf = 1;
    while (wpf & (wpf - 1)) wpf &= wpf - 1;    // a power of two
    const int ngroups = kFuseWarps / wpf;
    const int g = warp / wpf;
    const T* Sprev = (h & 1) ? Sbuf0 : Sbuf1;
    T* Scur = (h & 1) ? Sbuf1 : Sbuf0;
    const int slot = f.front_elems / ngroups;
    for (int k = beg + g; k < end; k += ngroups) {
      const int node = list[k];
      const NodeDev nd = f.a.nodes[node];
      T* Ssm = (h == L - 1) ? nullptr : Scur + f.fuse_soff[node];
      if (wpf == 1 && nd.nf <= 32) {
        warp_front<T>(f, node, nd, s, Sprev, Ssm);
      } else {
        const int t = threadIdx.x - g * wpf * 32;
        group_front<T>(f, node, nd, s, Sprev, Ssm, Fw + (size_t)g * slot, t, wpf * 32, 1 + g);
      }
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_subtree(const FuseArgs& f, int nroots, size_t smem_bytes, cudaStream_t st) {
  if (nroots == 0) return cudaSuccess;
  k_subtree<T><<<dim3(nroots, f.a.batch), kFuseWarps * 32, smem_bytes, st>>>(f);
  return cudaGetLastError();
}
template cudaError_t launch_subtree<double>(const FuseArgs&, int, size_t, cudaStream_t);
template cudaError_t launch_subtree<float>(const FuseArgs&, int, size_t, cudaStream_t);

cudaError_t configure_fused_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_subtree<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_subtree<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
