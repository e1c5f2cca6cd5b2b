// Right-hand-side sweep ("Leaves to Root" on a new load, Sec. 3.4 with the stored
// factors) and descent ("Root to Leaves", Eq. SchurC1 second line) over the bottom
// subtrees of the tree, one warp per (subtree, sample).
//
// The warp keeps the vertex values of the subtree's closed rectangle in shared memory:
// in the descent u (its border gathered once from the levels above, every interior
// value computed here and written back row by row at the end), in the sweep the load
// (read row by row at the start).  A node's boundary values and its sons' condensed
// loads therefore never leave the SM; the condensed loads wait on a per-warp stack
// (sons pushed in the sweep's order, taken by their father).  The factor store is laid
// out depth first, so a subtree's factor blocks (and y_g blocks) form one contiguous
// range per sample: the warp copies it into shared memory with 16-byte asynchronous
// copies (cp.async) issued at once, overlapped with the gather of the rectangle's
// values, and then solves node after node from shared memory.  The schedule and index
// maps of a subtree are the same for every sample: the CTA's warps serve kSubWarps
// samples of one subtree and share one copy of them.
//
// Per node (front rows r < nf - 1: r < m the eliminated vertices gamma, then B):
//   descent  t = y_g - L_Bg^T u_B, then L_gg^T u_g = t by columns from the last;
//   sweep    z = load at gamma + sons' condensed loads, then y_g = L_gg^-1 z_g column
//            by column with each column folded into the rows below it, leaving the
//            condensed load z_B - L_Bg y_g;
//   condensed leaves (G = K_gg^-1 and the boundary couplings w, see k_leaf.cu)
//            descent u_g = y_g - sum_i w_i u_B,i G[:, c_i]; sweep y_g = G z_g and
//            condensed load -w_i y_g[c_i].
#include "launch.h"

namespace hdd {

namespace {

constexpr unsigned kAll = 0xffffffffu;

struct SNode {
  int node, kind, m, b, nf, rec, y_off, f_rel, y_rel, b0, b1;
};

__device__ __forceinline__ SNode sched_at(const int32_t* e) {
  SNode q;
  q.node = e[0];
  const int w = e[1];
  q.kind = w & 3;
  q.m = (w >> 2) & 63;
  q.b = (w >> 8) & 4095;
  q.nf = (w >> 20) & 2047;
  q.rec = e[2];
  q.y_off = e[3];
  q.f_rel = e[4];
  q.y_rel = e[5];
  q.b0 = e[6];
  q.b1 = e[7];
  return q;
}

__device__ __forceinline__ int pad2(int n) { return (n + 1) & ~1; }
__device__ __forceinline__ int al16(int x) { return (x + 15) & ~15; }
// packed lower column-major index of (i, j), i >= j, of an m x m matrix
__device__ __forceinline__ int pk(int i, int j, int m) { return j * m - j * (j - 1) / 2 + (i - j); }

// A warp copies `bytes` (a multiple of 16) from global to shared memory, 16 bytes per
// lane and instruction, all in flight together (one commit group).
__device__ __forceinline__ void warp_copy16(void* dst, const void* src, int bytes, int lane) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const char* g = static_cast<const char*>(src);
  for (int o = 16 * lane; o < bytes; o += 512)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + o), "l"(g + o) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename T> __device__ __forceinline__ T* fac_of(const Arenas& A, int s);
template <> __device__ __forceinline__ double* fac_of<double>(const Arenas& A, int s) {
  return A.f64 + (int64_t)s * A.f64_stride;
}
template <> __device__ __forceinline__ float* fac_of<float>(const Arenas& A, int s) {
  return A.f32 + (int64_t)s * A.f32_stride;
}
template <typename T> __device__ __forceinline__ T* y_of(const Arenas& A, int s);
template <> __device__ __forceinline__ double* y_of<double>(const Arenas& A, int s) {
  return A.y64 + (int64_t)s * A.y64_stride;
}
template <> __device__ __forceinline__ float* y_of<float>(const Arenas& A, int s) {
  return A.y32 + (int64_t)s * A.y32_stride;
}
template <typename T> __device__ __forceinline__ T* s_of(const Arenas& A, int s);
template <> __device__ __forceinline__ double* s_of<double>(const Arenas& A, int s) {
  return A.s64 + (int64_t)s * A.s64_stride;
}
template <> __device__ __forceinline__ float* s_of<float>(const Arenas& A, int s) {
  return A.s32 + (int64_t)s * A.s32_stride;
}

// Sum of a[q] over the warp for q = 0..3 in six shuffles; lane l returns the sum for
// q = 2 * bit4(l) + bit3(l), so lane 8 q holds column q's.
template <typename T>
__device__ __forceinline__ T reduce4(const T (&a)[4], int lane) {
  const bool hi16 = lane & 16, hi8 = lane & 8;
  T x0 = hi16 ? a[2] : a[0], x1 = hi16 ? a[3] : a[1];
  const T y0 = hi16 ? a[0] : a[2], y1 = hi16 ? a[1] : a[3];
  x0 += __shfl_xor_sync(kAll, y0, 16);
  x1 += __shfl_xor_sync(kAll, y1, 16);
  T v = hi8 ? x1 : x0;
  const T o = hi8 ? x0 : x1;
  v += __shfl_xor_sync(kAll, o, 8);
  v += __shfl_xor_sync(kAll, v, 4);
  v += __shfl_xor_sync(kAll, v, 2);
  v += __shfl_xor_sync(kAll, v, 1);
  return v;
}

// Descent at a front (m <= 32 columns, nf - 1 <= 128 rows).  Lane c owns column c of
// the back substitution; lanes own rows lane + 32 j of the boundary product.
template <typename T>
__device__ __forceinline__ void descent_front(const SNode& q, const T* F, const T* Y, const int16_t* lm, T* region,
                                              int lane) {
  const int m = q.m, nr = q.nf - 1, ld = q.nf;
  if (m == 0) return;
  const int J = (nr + 31) >> 5;   // 32-row blocks of the front (at most 4)
  T w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = lane + 32 * j;
    w[j] = (j < J && r >= m && r < nr) ? region[lm[r]] : (T)0;
  }
  T t = (T)0;   // lane c: (L_Bg^T u_B)_c
  for (int c0 = 0; c0 < m; c0 += 4) {
    T acc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      acc[k] = (T)0;
      const int c = c0 + k;
      if (c < m) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (j >= J) break;   // uniform over the warp
          const int r = lane + 32 * j;
          if (r >= m && r < nr) acc[k] += F[c * ld + r] * w[j];
        }
      }
    }
    const T v = reduce4(acc, lane);
    const T tv = __shfl_sync(kAll, v, 8 * ((lane - c0) & 3));
    if (lane >= c0 && lane < c0 + 4) t = tv;
  }
  const T dinv = lane < m ? (T)1 / F[lane * ld + lane] : (T)0;
  t = lane < m ? Y[lane] - t : (T)0;
  for (int c = m - 1; c >= 0; --c) {
    const T uc = __shfl_sync(kAll, t * dinv, c);
    if (lane < c) t -= F[lane * ld + c] * uc;   // L_gg[c, lane]
    else if (lane == c) t = uc;
  }
  if (lane < m) region[lm[lane]] = t;
}

// Descent at a condensed leaf: lanes i < b first form w_i u_B,i and the coupled row c_i
// (shuffled to the others below); half-warp h then sums the boundary rows i = h, h + 2,
// ... for interior row r = lane & 15, reading G[r, c_i] through a column start that
// each lane keeps for its own row (the other one by a shuffle).
template <typename T>
__device__ __forceinline__ void descent_leaf(const SNode& q, const T* G, const T* Y, const int16_t* lm,
                                             const int16_t* cpl, T* region, int lane) {
  const int m = q.m, b = q.b;
  const T* wts = G + m * (m + 1) / 2;
  const int r = lane & 15;
  T twl[2];
  int cil[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {   // b <= 63: boundary rows lane and lane + 32
    const int i = lane + 32 * k;
    twl[k] = i < b ? wts[i] * region[lm[m + i]] : (T)0;
    cil[k] = i < b ? cpl[i] : -1;
  }
  const int cs = r * m - r * (r - 1) / 2 - r;   // packed index of (i, r), i >= r: cs + i
  T acc = (T)0;
  for (int i0 = 0; i0 < b; i0 += 2) {   // same trip count in both halves (the shuffles)
    const int i = i0 + (lane >> 4);       // i0 is even: i and i0 lie on the same side of 32
    const int src = i & 31;
    const T tw = __shfl_sync(kAll, i0 < 32 ? twl[0] : twl[1], src);
    const int cix = __shfl_sync(kAll, i0 < 32 ? cil[0] : cil[1], src);
    const int ci = i < b ? cix : -1;
    const int csc = __shfl_sync(kAll, cs, ci >= 0 ? ci : 0);
    if (r < m && ci >= 0) acc += tw * G[r >= ci ? csc + r : cs + ci];
  }
  acc += __shfl_xor_sync(kAll, acc, 16);
  __syncwarp();
  if (lane < m) region[lm[lane]] = Y[lane] - acc;
}

// Right-hand-side sweep at a front: z from the load and the sons' condensed loads (the
// top two entries of the stack: son 0's on top), forward substitution, y_g out, the
// condensed load onto the stack (or to the Schur block's start for the subtree root).
template <typename T>
__device__ __forceinline__ void sweep_front(const SNode& q, const T* F, const int16_t* lm, const T* region, T* stack,
                                            int& sp, T* Yg, T* Sroot, int lane) {
  const int m = q.m, nr = q.nf - 1, ld = q.nf;
  const T* cond0 = stack + sp - q.b0;
  const T* cond1 = cond0 - q.b1;
  const int16_t* p0 = lm + pad2(nr);
  const int16_t* p1 = p0 + pad2(nr);
  const int J = (nr + 31) >> 5;   // 32-row blocks of the front (at most 4)
  T z[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = lane + 32 * j;
    T v = (T)0;
    if (j < J && r < nr) {
      if (r < m) v = region[lm[r]];
      if (q.kind == 0) {
        const int a = p0[r], c = p1[r];
        if (a >= 0) v += cond0[a];
        if (c >= 0) v += cond1[c];
      }
    }
    z[j] = v;
  }
  const T dinv = lane < m ? (T)1 / F[lane * ld + lane] : (T)0;
  for (int c = 0; c < m; ++c) {
    if (lane == c) z[0] *= dinv;
    const T yc = __shfl_sync(kAll, z[0], c);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (j >= J) break;   // uniform over the warp
      const int r = lane + 32 * j;
      if (r > c && r < nr) z[j] -= F[c * ld + r] * yc;
    }
  }
  if (lane < m) Yg[q.y_off + lane] = z[0];
  __syncwarp();   // the sons' loads are read: their stack space takes this node's
  const int base = q.kind == 0 ? sp - q.b0 - q.b1 : sp;
  T* out = Sroot ? Sroot : stack + base;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int r = lane + 32 * j;
    if (j < J && r >= m && r < nr) out[r - m] = z[j];
  }
  sp = Sroot ? base : base + q.b;
}

// Right-hand-side sweep at a condensed leaf.
template <typename T>
__device__ __forceinline__ void sweep_leaf(const SNode& q, const T* G, const int16_t* lm, const int16_t* cpl,
                                           const T* region, T* stack, int& sp, T* Yg, T* Sroot, int lane) {
  const int m = q.m, b = q.b;
  const T* wts = G + m * (m + 1) / 2;
  // y = G z: half-warp h sums the columns j = h, h + 2, ... for row r = lane & 15, reading
  // G[r, j] through a column start that each lane keeps for its own row (the other by a
  // shuffle); the halves' sums are then added
  const int r = lane & 15;
  const T zr = lane < m ? region[lm[lane]] : (T)0;
  const int cs = r * m - r * (r - 1) / 2 - r;   // packed index of (i, r), i >= r: cs + i
  T y = (T)0;
  for (int j0 = 0; j0 < m; j0 += 2) {   // same trip count in both halves (the shuffles)
    const int j = j0 + (lane >> 4);
    const int jj = j < m ? j : 0;
    const T zj = __shfl_sync(kAll, zr, jj);
    const int csj = __shfl_sync(kAll, cs, jj);
    if (r < m && j < m) y += G[r >= j ? csj + r : cs + j] * zj;
  }
  y += __shfl_xor_sync(kAll, y, 16);   // lanes r and r + 16 both hold row r's sum
  if (lane < m) Yg[q.y_off + lane] = y;
  T* out = Sroot ? Sroot : stack + sp;
  for (int i0 = 0; i0 < b; i0 += 32) {
    const int i = i0 + lane;
    const int ci = i < b ? cpl[i] : -1;
    const T yc = __shfl_sync(kAll, y, ci >= 0 ? ci : 0);
    if (i < b) out[i] = ci >= 0 ? -wts[i] * yc : (T)0;
  }
  if (!Sroot) sp += b;
}

// Shared memory of a CTA: the subtree's schedule and maps, then per warp its part
// (descent: factor range, y_g range, rectangle; sweep: factor range, rectangle, stack).
struct SubSmem {
  int32_t* sched;
  int16_t* rec;
  unsigned char* warp;
};

__device__ __forceinline__ SubSmem sub_setup(const SubArgs& g, unsigned char* smem, const int32_t* D, int warp) {
  SubSmem sm;
  sm.sched = reinterpret_cast<int32_t*>(smem);
  sm.rec = reinterpret_cast<int16_t*>(smem + g.sched_bytes);
  const int n = D[1];
  const int32_t* src = g.sched + (int64_t)D[0] * kSchedInts;
  for (int i = threadIdx.x; i < n * kSchedInts; i += blockDim.x) sm.sched[i] = src[i];
  const int32_t* rsrc = reinterpret_cast<const int32_t*>(g.rec + D[2]);
  int32_t* rdst = reinterpret_cast<int32_t*>(sm.rec);
  for (int i = threadIdx.x; i < D[3] / 2; i += blockDim.x) rdst[i] = rsrc[i];
  sm.warp = smem + g.sched_bytes + g.rec_bytes + (size_t)warp * g.warp_bytes;
  return sm;
}

__device__ __forceinline__ int64_t sub_f_off(const int32_t* D) {
  return (int64_t)(uint32_t)D[8] | ((int64_t)D[9] << 32);
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(32 * kSubWarps) k_descent_sub(SubArgs g, double* __restrict__ u, int64_t u_stride) {
  const int32_t* D = g.subs + (int64_t)blockIdx.x * kSubInts;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubSmem sm = sub_setup(g, smem_raw, D, warp);
  __syncthreads();
  const int s = blockIdx.y * kSubWarps + warp;
  if (s >= g.batch) return;
  const int n = D[1], x0 = D[4], y0 = D[5], w = D[6], h = D[7];
  T* Fs = reinterpret_cast<T*>(sm.warp);
  T* Ys = reinterpret_cast<T*>(sm.warp + g.fac_bytes);
  T* region = reinterpret_cast<T*>(sm.warp + g.fac_bytes + g.y_bytes);
  warp_copy16(Fs, fac_of<T>(g.A, s) + sub_f_off(D), al16(D[10] * (int)sizeof(T)), lane);
  warp_copy16(Ys, y_of<T>(g.A, s) + D[11], al16(D[12] * (int)sizeof(T)), lane);
  cp_commit();
  double* us = u + (int64_t)s * u_stride;
  {   // the root's boundary values, from the levels above
    const SNode q = sched_at(sm.sched);
    const int32_t* vid = g.maps + g.nodes[q.node].map_off;
    const int16_t* lm = sm.rec + q.rec;
    for (int i = lane; i < q.b; i += 32) region[lm[q.m + i]] = (T)us[vid[q.m + i]];
  }
  cp_wait_all();
  __syncwarp();
  for (int k = 0; k < n; ++k) {
    const SNode q = sched_at(sm.sched + kSchedInts * k);
    const int16_t* lm = sm.rec + q.rec;
    if (q.kind == 2)
      descent_leaf<T>(q, Fs + q.f_rel, Ys + q.y_rel, lm, lm + pad2(q.nf - 1), region, lane);
    else
      descent_front<T>(q, Fs + q.f_rel, Ys + q.y_rel, lm, region, lane);
    __syncwarp();
  }
  for (int yy = 1; yy < h - 1; ++yy)
    for (int xx = 1 + lane; xx < w - 1; xx += 32)
      us[(int64_t)(y0 + yy) * g.N + x0 + xx] = (double)region[yy * w + xx];
}

template <typename T>
__global__ void __launch_bounds__(32 * kSubWarps) k_forward_sub(SubArgs g, Rhs rhs) {
  const int32_t* D = g.subs + (int64_t)blockIdx.x * kSubInts;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SubSmem sm = sub_setup(g, smem_raw, D, warp);
  __syncthreads();
  const int s = blockIdx.y * kSubWarps + warp;
  if (s >= g.batch) return;
  const int n = D[1], x0 = D[4], y0 = D[5], w = D[6], h = D[7];
  T* Fs = reinterpret_cast<T*>(sm.warp);
  T* region = reinterpret_cast<T*>(sm.warp + g.fac_bytes);
  T* stack = reinterpret_cast<T*>(sm.warp + g.fac_bytes + g.region_bytes);
  warp_copy16(Fs, fac_of<T>(g.A, s) + sub_f_off(D), al16(D[10] * (int)sizeof(T)), lane);
  cp_commit();
  for (int yy = 1; yy < h - 1; ++yy)
    for (int xx = 1 + lane; xx < w - 1; xx += 32) region[yy * w + xx] = (T)rhs(s, (y0 + yy) * g.N + x0 + xx);
  cp_wait_all();
  __syncwarp();
  T* Yg = y_of<T>(g.A, s);
  T* Sroot = s_of<T>(g.A, s) + g.nodes[sched_at(sm.sched).node].s_off;
  int sp = 0;
  for (int k = n - 1; k >= 0; --k) {
    const SNode q = sched_at(sm.sched + kSchedInts * k);
    const int16_t* lm = sm.rec + q.rec;
    T* root_out = k == 0 ? Sroot : nullptr;
    if (q.kind == 2)
      sweep_leaf<T>(q, Fs + q.f_rel, lm, lm + pad2(q.nf - 1), region, stack, sp, Yg, root_out, lane);
    else
      sweep_front<T>(q, Fs + q.f_rel, lm, region, stack, sp, Yg, root_out, lane);
    __syncwarp();
  }
}

template <typename T>
cudaError_t launch_descent_sub(const SubArgs& g, int n_sub, size_t smem, double* u, int64_t u_stride,
                               cudaStream_t st) {
  if (n_sub == 0 || g.batch == 0) return cudaSuccess;
  const dim3 grid(n_sub, (g.batch + kSubWarps - 1) / kSubWarps);
  k_descent_sub<T><<<grid, 32 * kSubWarps, smem, st>>>(g, u, u_stride);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_forward_sub(const SubArgs& g, int n_sub, size_t smem, const Rhs& rhs, cudaStream_t st) {
  if (n_sub == 0 || g.batch == 0) return cudaSuccess;
  const dim3 grid(n_sub, (g.batch + kSubWarps - 1) / kSubWarps);
  k_forward_sub<T><<<grid, 32 * kSubWarps, smem, st>>>(g, rhs);
  return cudaGetLastError();
}
template cudaError_t launch_descent_sub<double>(const SubArgs&, int, size_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_descent_sub<float>(const SubArgs&, int, size_t, double*, int64_t, cudaStream_t);
template cudaError_t launch_forward_sub<double>(const SubArgs&, int, size_t, const Rhs&, cudaStream_t);
template cudaError_t launch_forward_sub<float>(const SubArgs&, int, size_t, const Rhs&, cudaStream_t);

cudaError_t configure_sweep_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_descent_sub<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_descent_sub<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_forward_sub<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_forward_sub<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
