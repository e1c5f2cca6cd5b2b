// Fronts of up to kSmallMax rows ("Leaves to Root", Sec. 3.4), W warps per
// front.  A CTA serves G = (CTA warps) / W consecutive samples of one node, so
// the node's index tables are staged once per CTA and each group of W warps
// owns one front in shared memory (column-major, leading dimension ld).
//
// Per front:
//   1. build: leaves from the five-point stencil of their own triangles (the P1
//      element matrix of Eq. coefA on this mesh; only the nonzeros are written),
//      fathers by adding the sons' lower Schur triangles through their up maps
//      (Sec. 3.3, Eq. block_equation4);
//   2. left-looking Cholesky of the m gamma columns, which also turns the
//      bordered right-hand-side row into y_g^T (the father's gamma load is added
//      to that row when its column is first touched);
//   3. S = K_BB - L_Bg L_Bg^T (Eq. SchurC1) in 4 x 4 register tiles, written
//      straight to the node's Schur block, and the factor columns F = [L_gg;
//      L_Bg; y_g^T] to the factor store.
// Barriers are per group (a warp barrier when W = 1), so the groups of a CTA
// never wait for one another.
#include "launch.h"

namespace hdd {

namespace {

template <typename T> __device__ __forceinline__ T* grp_F(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* grp_F<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ float* grp_F<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}
template <typename T> __device__ __forceinline__ T* grp_S(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ double* grp_S<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s64 + (int64_t)s * A.s64_stride + nd.s_off;
}
template <> __device__ __forceinline__ float* grp_S<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.s32 + (int64_t)s * A.s32_stride + nd.s_off;
}

__device__ __forceinline__ void ld4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Lower-triangle tile (ti >= tj) of linear index t, enumerated column by column
// (tile column tj holds nt - tj tiles), so that consecutive t walk down a column.
__device__ __forceinline__ void tile_of(int t, int nt, int& ti, int& tj) {
  const int u = nt * (nt + 1) / 2 - 1 - t;   // row-major lower index, reversed
  int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > u) --r;
  while ((r + 1) * (r + 2) / 2 <= u) ++r;
  const int c = u - r * (r + 1) / 2;
  tj = nt - 1 - r;
  ti = nt - 1 - c;
}

// Barrier of one group.  A CTA holds at most two groups of more than one warp,
// which use the named barriers 1 and 2 (constant ids: the SM's barrier budget
// per CTA is what the kernel names, and it bounds the CTAs per SM).
template <int W>
struct Group {
  static constexpr int size = 32 * W;   // threads of the group (W warps)
  int id, t;                            // named barrier id (1 or 2), thread index in the group
  __device__ __forceinline__ void sync() const {
    if (W == 1) __syncwarp();
    else if (id == 1) asm volatile("bar.sync 1, %0;" ::"n"(size) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"n"(size) : "memory");
  }
};

// Adds a son's lower Schur triangle ((b+1) x (b+1), column-major) into the front
// through its up map ups (son row -> front row).  The triangle of n = b + 1 columns
// is walked as ceil(n / 2) folded columns of n + 1 entries (column c followed by
// column n - 1 - c, which together hold n + 1 entries; for odd n the middle column
// stands alone), so entry e of the walk maps to its (row, column) without a loop;
// four entries per pass, loads first.
template <typename T, class Grp>
__device__ __forceinline__ void add_son(T* K, int ld, const NodeDev& ch, const int* ups, const Arenas& A, int s,
                                        const Grp& g) {
  const int n = ch.b + 1;
  const int total = n * (n + 1) / 2;
  const int64_t base = (int64_t)s * (ch.fp64 ? A.s64_stride : A.s32_stride) + ch.s_off;
  const float inv_w = 1.0f / (float)(n + 1);
  for (int i0 = g.t; i0 < total; i0 += 4 * g.size) {
    T v[4];
    int rr[4], cc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = i0 + q * g.size;
      int f = (int)((float)e * inv_w);   // folded column, corrected for rounding
      if (f * (n + 1) > e) --f;
      if ((f + 1) * (n + 1) <= e) ++f;
      const int p = e - f * (n + 1);
      const bool first = p < n - f;      // in column f, else in column n - 1 - f
      cc[q] = first ? f : n - 1 - f;
      rr[q] = first ? f + p : cc[q] + (p - (n - f));
      const bool use = e < total;
      const int64_t at = base + (int64_t)cc[q] * n + rr[q];
      v[q] = use ? (ch.fp64 ? (T)A.s64[at] : (T)A.s32[at]) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (i0 + q * g.size < total) {
        const int pr = ups[rr[q]], pc = ups[cc[q]];
        K[min(pr, pc) * ld + max(pr, pc)] += v[q];
      }
    }
  }
}

}  // namespace

// MP: the launch covers several plans (the per-plan fields are bound per CTA; a
// separate instantiation keeps the single-plan kernel's registers as they are)
template <typename T, int W, bool MP>
__global__ void __launch_bounds__(256) k_front_group(StepArgs a, int ld, int fr_elems) {
  const int node = a.list[blockIdx.x];
  if (MP) bind_plan(a, node);
  const NodeDev nd = a.nodes[node];
  const int nf = nd.nf, m = nd.m, nb = nd.b + 1, N = a.N;
  const int G = (blockDim.x >> 5) / W;
  const int gi = (threadIdx.x >> 5) / W;
  const Group<W> g{1 + gi, (int)threadIdx.x - gi * 32 * W};
  const int s = blockIdx.y * G + gi;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* K = reinterpret_cast<T*>(smem_raw) + (size_t)gi * fr_elems;
  T* dg = K + (size_t)((nf + 3) & ~3) * ld;   // pivots sqrt(p_k) of this front
  int* sh = reinterpret_cast<int*>(reinterpret_cast<T*>(smem_raw) + (size_t)G * fr_elems);
  const int32_t* map = a.maps + nd.map_off;

  // node tables, once per CTA: leaf -> front row of each vertex of its closed
  // rectangle (-1: Dirichlet); father -> the sons' up maps
  const int tw = nd.x1 - nd.x0 + 1;
  NodeDev c0{}, c1{};
  if (nd.leaf) {
    const int cells = tw * (nd.y1 - nd.y0 + 1);
    for (int i = threadIdx.x; i < cells; i += blockDim.x) sh[i] = -1;
    __syncthreads();
    int* loc = sh + cells;   // per front row: local (column, row) of its vertex, 16 bits each
    for (int r = threadIdx.x; r < nf - 1; r += blockDim.x) {
      const int v = map[r];
      const int li = v % N - nd.x0, lj = v / N - nd.y0;
      sh[lj * tw + li] = r;
      loc[r] = (lj << 16) | li;
    }
  } else {
    c0 = a.nodes[nd.child0];
    c1 = a.nodes[nd.child1];
    const int32_t* up0 = a.maps + c0.up_off;
    const int32_t* up1 = a.maps + c1.up_off;
    for (int i = threadIdx.x; i <= c0.b; i += blockDim.x) sh[i] = up0[i];
    for (int i = threadIdx.x; i <= c1.b; i += blockDim.x) sh[c0.b + 1 + i] = up1[i];
  }
  __syncthreads();
  if (s >= a.batch) return;

  // 1. build (the front is zero outside its lower triangle's nonzeros)
  {
    const int n16 = (int)(((size_t)((nf + 3) & ~3) * ld * sizeof(T)) / 16);
    uint4* z = reinterpret_cast<uint4*>(K);
    for (int i = g.t; i < n16; i += g.size) z[i] = make_uint4(0, 0, 0, 0);
  }
  g.sync();
  if (nd.leaf) {
    const T* kap = kappa_of<T>(a.kappa, a.kappa32) + (int64_t)s * a.kap_stride;
    const int* loc = sh + tw * (nd.y1 - nd.y0 + 1);
    for (int r = g.t; r < nf - 1; r += g.size) {
      const int li = loc[r] & 0xffff, lj = loc[r] >> 16;
      const int vi = nd.x0 + li, vj = nd.y0 + lj;
      const T wl = w_horizontal(kap, N, nd, vi - 1, vj), wr = w_horizontal(kap, N, nd, vi, vj);
      const T wd = w_vertical(kap, N, nd, vi, vj - 1), wu = w_vertical(kap, N, nd, vi, vj);
      K[r * ld + r] = wl + wr + wd + wu;
      // couplings to neighbours of a smaller front row: entry (r, c), r > c
      if (li > 0) { const int c = sh[lj * tw + li - 1]; if (c >= 0 && c < r) K[c * ld + r] = -wl; }
      if (vi < nd.x1) { const int c = sh[lj * tw + li + 1]; if (c >= 0 && c < r) K[c * ld + r] = -wr; }
      if (lj > 0) { const int c = sh[(lj - 1) * tw + li]; if (c >= 0 && c < r) K[c * ld + r] = -wd; }
      if (vj < nd.y1) { const int c = sh[(lj + 1) * tw + li]; if (c >= 0 && c < r) K[c * ld + r] = -wu; }
      if (r < m) K[r * ld + nf - 1] = (T)a.rhs(s, vj * N + vi);   // load of an interior vertex (Eq. coefc)
    }
  } else {
    add_son<T>(K, ld, c0, sh, a.arenas, s, g);
    g.sync();
    add_son<T>(K, ld, c1, sh + c0.b + 1, a.arenas, s, g);
  }
  g.sync();

  // 2. left-looking Cholesky of the gamma columns in blocks of four; rows are spread
  // over the group.  A block's columns first take the products with every column to
  // its left (one 16-byte load of the four columns' entries per row entry), then, one
  // by one, the products within the block, each column's products summed before they
  // are subtracted from its entries: the entry is usually much larger than what is
  // left of it, and few roundings at its magnitude are enough.
  bool bad = false;
  for (int kb = 0; kb < m; kb += 4) {
    const int nbk = min(4, m - kb);
    for (int r = kb + g.t; r < nf; r += g.size) {
      T dot[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll 2
      for (int l = 0; l < kb; ++l) {
        const T x = K[l * ld + r];
        T y[4];
        ld4(K + l * ld + kb, y);   // entries (kb .. kb + 3, l)
#pragma unroll
        for (int q = 0; q < 4; ++q) dot[q] += x * y[q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = kb + q;
        if (q < nbk && r >= k) {
          T acc = K[k * ld + r];
          if (r == nf - 1 && !nd.leaf) acc += (T)a.rhs(s, map[k]);   // father: load of its gamma vertex
          K[k * ld + r] = acc - dot[q];
        }
      }
    }
    g.sync();
    for (int q = 0; q < nbk; ++q) {
      const int k = kb + q;
      if (q > 0) {   // products with the block's earlier columns
        for (int r = k + g.t; r < nf; r += g.size) {
          T dot = (T)0;
          for (int l = kb; l < k; ++l) dot += K[l * ld + r] * K[l * ld + k];
          K[k * ld + r] -= dot;
        }
        g.sync();
      }
      T p = K[k * ld + k];
      if (!(p > (T)0) || !isfinite(p)) {   // not SPD: record, continue with a unit pivot
        bad = true;
        p = (T)1;
      }
      const T d = sqrt(p), inv = (T)1 / d;
      for (int r = k + 1 + g.t; r < nf; r += g.size) K[k * ld + r] *= inv;
      if (g.t == 0) dg[k] = d;
      g.sync();
    }
  }
  if (bad && g.t == 0) flag_status(a.status, s, -HDD_ENOTSPD, node);

  // 3a. factor columns and y_g
  T* F = grp_F<T>(a.arenas, nd, s);
  for (int c = 0; c < m; ++c)
    for (int r = g.t; r < nf; r += g.size) F[c * nf + r] = (r == c) ? dg[c] : K[c * ld + r];
  T* Y = node_Y<T>(a.arenas, nd, s);
  for (int c = g.t; c < m; c += g.size) Y[c] = K[c * ld + nf - 1];

  // 3b. Schur block over 4 x 4 tiles aligned to multiples of 4 front rows
  T* S = grp_S<T>(a.arenas, nd, s);
  const int t0 = m & ~3;
  const int nt = (nf - t0 + 3) >> 2;
  const int ntiles = nt * (nt + 1) / 2;
  for (int t = g.t; t < ntiles; t += g.size) {
    int ti, tj;
    tile_of(t, nt, ti, tj);
    const int i0 = t0 + 4 * ti, j0 = t0 + 4 * tj;
    T acc[4][4];   // L_Bg L_Bg^T, summed before it is subtracted from the front's entries
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[q][w] = (T)0;
#pragma unroll 2
    for (int l = 0; l < m; ++l) {
      T x[4], y[4];
      ld4(K + l * ld + i0, x);
      ld4(K + l * ld + j0, y);
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] += x[q] * y[w];
    }
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const int c = j0 + w;
      if (c < m || c >= nf) continue;
      T kv[4];   // the front's boundary-block entries
      ld4(K + c * ld + i0, kv);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = i0 + q;
        if (r >= c && r < nf) S[(c - m) * nb + (r - m)] = kv[q] - acc[q][w];
      }
    }
  }
}

// Warps per front: enough that a group's rows and tiles keep its lanes busy,
// few enough that several fronts share a CTA.
int group_warps(int max_nf, bool fp64) {
  if (max_nf <= 48) return 1;
  if (max_nf <= 64) return 2;
  if (!fp64 || max_nf <= 128) return 4;
  return 8;
}

static int group_ld(int nf) {   // multiple of 4, congruent to 4 modulo 8
  int ld = (nf + 3) & ~3;
  if ((ld & 7) == 0) ld += 4;
  return ld;
}

template <typename T>
cudaError_t launch_front_group(const StepArgs& a, int family, cudaStream_t st) {
  if (a.nlist == 0) return cudaSuccess;
  const int W = group_warps(a.max_nf, sizeof(T) == 8);
  const int warps = W > 4 ? W : 4;
  const int G = warps / W;
  const int ld = group_ld(a.max_nf);
  const int fr_elems = (((a.max_nf + 3) & ~3) * ld + a.max_m + 3) & ~3;
  const int ints = max(a.max_rect + a.max_nf, 2 * a.max_nf + 2);
  const size_t smem = (size_t)G * fr_elems * sizeof(T) + (size_t)ints * sizeof(int);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  dim3 grid(a.nlist, (a.batch + G - 1) / G);
  if (a.prof) a.prof->begin(family, a.fl_chol + a.fl_trsm + a.fl_syrk + a.fl_rhs, st);
  if (a.plan_of) {
    switch (W) {
      case 1: k_front_group<T, 1, true><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      case 2: k_front_group<T, 2, true><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      case 4: k_front_group<T, 4, true><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      default: k_front_group<T, 8, true><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
    }
  } else {
    switch (W) {
      case 1: k_front_group<T, 1, false><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      case 2: k_front_group<T, 2, false><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      case 4: k_front_group<T, 4, false><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
      default: k_front_group<T, 8, false><<<grid, warps * 32, smem, st>>>(a, ld, fr_elems); break;
    }
  }
  if (a.prof) a.prof->end(st);
  return cudaGetLastError();
}
template cudaError_t launch_front_group<double>(const StepArgs&, int, cudaStream_t);
template cudaError_t launch_front_group<float>(const StepArgs&, int, cudaStream_t);

cudaError_t configure_group_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  // the whole unified L1 / shared-memory array as shared memory: the residency of
  // these CTAs is bounded by their fronts, not by L1
  const void* fns[] = {
      (const void*)k_front_group<double, 1, false>, (const void*)k_front_group<double, 2, false>,
      (const void*)k_front_group<double, 4, false>, (const void*)k_front_group<double, 8, false>,
      (const void*)k_front_group<float, 1, false>,  (const void*)k_front_group<float, 2, false>,
      (const void*)k_front_group<float, 4, false>,  (const void*)k_front_group<float, 8, false>,
      (const void*)k_front_group<double, 1, true>,  (const void*)k_front_group<double, 2, true>,
      (const void*)k_front_group<double, 4, true>,  (const void*)k_front_group<double, 8, true>,
      (const void*)k_front_group<float, 1, true>,   (const void*)k_front_group<float, 2, true>,
      (const void*)k_front_group<float, 4, true>,   (const void*)k_front_group<float, 8, true>};
  for (const void* f : fns) {
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared)))
      return e;
  }
  return cudaSuccess;
}

}  // namespace hdd
