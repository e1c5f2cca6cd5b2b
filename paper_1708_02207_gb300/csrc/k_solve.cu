// Assembly of kappa, the pruned descent and the misfit.
#include "launch.h"

namespace hdd {

// ---------------------------------------------------------------------------
// Assembly (Sec. 3.1; notation table: kappa = e^q): q[s,t] = sum_k Phi[t,k] Z[s,k]
// accumulated in k order, kappa = exp(q), FP64.  CTA = 128 triangles x 8 samples;
// Phi and Z chunks staged in shared memory, Phi read once per 8 samples.
constexpr int kKapT = 128, kKapS = 8, kKapK = 32;

__global__ void k_kappa(const double* __restrict__ phi, const double* __restrict__ Z, int n_t, int n_z, int batch,
                        double* __restrict__ kappa, float* __restrict__ kappa32, int64_t kap_stride) {
  __shared__ double ph[kKapK][kKapT + 1];
  __shared__ double zs[kKapS][kKapK];
  const int t0 = blockIdx.x * kKapT, s0 = blockIdx.y * kKapS;
  const int t = t0 + threadIdx.x;
  double acc[kKapS];
#pragma unroll
  for (int q = 0; q < kKapS; ++q) acc[q] = 0.0;
  for (int k0 = 0; k0 < n_z; k0 += kKapK) {
    const int kc = min(kKapK, n_z - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kKapT * kc; e += blockDim.x) {
      const int tt = e / kc, kk = e - tt * kc;
      ph[kk][tt] = (t0 + tt < n_t) ? phi[(int64_t)(t0 + tt) * n_z + k0 + kk] : 0.0;
    }
    for (int e = threadIdx.x; e < kKapS * kc; e += blockDim.x) {
      const int ss = e / kc, kk = e - ss * kc;
      zs[ss][kk] = (s0 + ss < batch) ? Z[(int64_t)(s0 + ss) * n_z + k0 + kk] : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const double p = ph[kk][threadIdx.x];
#pragma unroll
      for (int q = 0; q < kKapS; ++q) acc[q] = fma(p, zs[q][kk], acc[q]);
    }
  }
  if (t < n_t) {
#pragma unroll
    for (int q = 0; q < kKapS; ++q)
      if (s0 + q < batch) {
        const double kv = exp(acc[q]);
        kappa[(int64_t)(s0 + q) * kap_stride + t] = kv;
        if (kappa32) kappa32[(int64_t)(s0 + q) * kap_stride + t] = (float)kv;
      }
  }
}

// ---------------------------------------------------------------------------
// Assembly for mixed-precision plans without the FP64 pipe: q = sum_k Phi Z and
// kappa = exp(q) in double-float arithmetic (pairs of FP32 values, hi + lo, ~48
// significant bits), with the error-free transformations TwoSum (Knuth) and
// TwoProduct via FMA (Dekker's product).  exp uses the additive range reduction
// q = k ln2 + r (ln2 as a hi/lo pair, the product k ln2 formed exactly) and the
// Taylor series of e^r to degree 12 (|r| <= ln2/2, remainder < 2e-16) in
// Horner form; e^q = 2^k e^r.  Outputs the FP64 kappa (residual) and its FP32
// copy (factorisation).
namespace {
struct dflt { float hi, lo; };
__device__ __forceinline__ dflt qsum(float a, float b) { const float s = a + b; return {s, b - (s - a)}; }
__device__ __forceinline__ dflt tsum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dflt df_add(dflt a, dflt b) {
  dflt s = tsum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return qsum(s.hi, s.lo);
}
__device__ __forceinline__ dflt df_mul(dflt a, dflt b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return qsum(p, e);
}
// 1/n! as hi + lo pairs (the FP32 value nearest to 1/n!, then the nearest to the rest)
__constant__ float kInvFact[13][2] = {
    {1.0f, 0.0f}, {1.0f, 0.0f}, {0.5f, 0.0f},
    {0.1666666716337204f, -4.967053879312289e-09f}, {0.0416666679084301f, -1.2417634698280722e-09f},
    {0.008333333767950535f, -4.34617203337595e-10f}, {0.0013888889225199819f, -3.3631094437103215e-11f},
    {0.00019841270113829523f, -2.725596874933456e-12f}, {2.4801587642286904e-05f, -3.40699609366682e-13f},
    {2.7557318844628753e-06f, 3.793571224297229e-14f}, {2.755731998149713e-07f, -7.575112209051195e-15f},
    {2.5052107943679403e-08f, 4.4176230446483665e-16f}, {2.0876755879584152e-09f, 1.1082839147459852e-16f}};
// ln 2 as hi + lo
constexpr float kLn2Hi = 0.6931471824645996f, kLn2Lo = -1.9046542121259336e-09f;

__device__ __forceinline__ dflt df_exp(dflt q, int* k_out) {
  const float kf = rintf(q.hi * 1.4426950408889634f);
  dflt kl = {kf * kLn2Hi, 0.0f};
  kl.lo = fmaf(kf, kLn2Hi, -kl.hi);          // k ln2_hi exactly, as hi + lo
  kl.lo = fmaf(kf, kLn2Lo, kl.lo);
  const dflt r = df_add(q, dflt{-kl.hi, -kl.lo});
  dflt p = {kInvFact[12][0], kInvFact[12][1]};
#pragma unroll
  for (int n = 11; n >= 0; --n) p = df_add(df_mul(p, r), dflt{kInvFact[n][0], kInvFact[n][1]});
  *k_out = (int)kf;
  return p;
}
}  // namespace

__global__ void k_kappa_df(const float* __restrict__ phi_hi, const float* __restrict__ phi_lo,
                           const double* __restrict__ Z, int n_t, int n_z, int batch, double* __restrict__ kappa,
                           float* __restrict__ kappa32, int64_t kap_stride) {
  __shared__ float ph[kKapK][kKapT + 1], pl[kKapK][kKapT + 1];
  __shared__ float zh[kKapS][kKapK], zl[kKapS][kKapK];
  const int t0 = blockIdx.x * kKapT, s0 = blockIdx.y * kKapS;
  const int t = t0 + threadIdx.x;
  float ah[kKapS], al[kKapS];
#pragma unroll
  for (int q = 0; q < kKapS; ++q) ah[q] = al[q] = 0.0f;
  for (int k0 = 0; k0 < n_z; k0 += kKapK) {
    const int kc = min(kKapK, n_z - k0);
    __syncthreads();
    for (int e = threadIdx.x; e < kKapT * kc; e += blockDim.x) {
      const int tt = e / kc, kk = e - tt * kc;
      const bool in = t0 + tt < n_t;
      ph[kk][tt] = in ? phi_hi[(int64_t)(t0 + tt) * n_z + k0 + kk] : 0.0f;
      pl[kk][tt] = in ? phi_lo[(int64_t)(t0 + tt) * n_z + k0 + kk] : 0.0f;
    }
    for (int e = threadIdx.x; e < kKapS * kc; e += blockDim.x) {
      const int ss = e / kc, kk = e - ss * kc;
      const double z = (s0 + ss < batch) ? Z[(int64_t)(s0 + ss) * n_z + k0 + kk] : 0.0;
      const float h = (float)z;
      zh[ss][kk] = h;
      zl[ss][kk] = (float)(z - (double)h);
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const float a = ph[kk][threadIdx.x], b = pl[kk][threadIdx.x];
#pragma unroll
      for (int q = 0; q < kKapS; ++q) {
        const float zq = zh[q][kk];
        const float p = a * zq;
        float e = fmaf(a, zq, -p);
        e = fmaf(a, zl[q][kk], fmaf(b, zq, e));
        const dflt s = tsum(ah[q], p);     // (ah, al) += (p, e)
        ah[q] = s.hi;
        al[q] += s.lo + e;
      }
    }
  }
  if (t < n_t) {
#pragma unroll
    for (int q = 0; q < kKapS; ++q) {
      if (s0 + q >= batch) continue;
      int k;
      const dflt ex = df_exp(qsum(ah[q], al[q]), &k);
      const double scale = k > 1023 ? (double)INFINITY
                                    : (k < -1022 ? 0.0 : __longlong_as_double((long long)(1023 + k) << 52));   // 2^k
      kappa[(int64_t)(s0 + q) * kap_stride + t] = ((double)ex.hi + (double)ex.lo) * scale;
      kappa32[(int64_t)(s0 + q) * kap_stride + t] = ldexpf(ex.hi, k);
    }
  }
}

cudaError_t launch_kappa_df(const float* phi_hi, const float* phi_lo, const double* Z, int n_t, int n_z, int batch,
                            double* kappa, float* kappa32, int64_t kap_stride, cudaStream_t st) {
  dim3 grid((n_t + kKapT - 1) / kKapT, (batch + kKapS - 1) / kKapS);
  k_kappa_df<<<grid, kKapT, 0, st>>>(phi_hi, phi_lo, Z, n_t, n_z, batch, kappa, kappa32, kap_stride);
  return cudaGetLastError();
}

cudaError_t launch_kappa(const double* phi, const double* Z, int n_t, int n_z, int batch, double* kappa,
                         float* kappa32, int64_t kap_stride, cudaStream_t st) {
  dim3 grid((n_t + kKapT - 1) / kKapT, (batch + kKapS - 1) / kKapS);
  k_kappa<<<grid, kKapT, 0, st>>>(phi, Z, n_t, n_z, batch, kappa, kappa32, kap_stride);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// "Root to Leaves" at one node (Sec. 3.4; Eq. SchurC1 second line,
// u_2 = A22^-1 F2 c - A22^-1 A21 u_1): with the stored partial Cholesky factors
//   t = y_g - L_Bg^T u_B,   L_gg^T u_g = t.
// One CTA per (node, sample).  t by one warp per column (coalesced down the
// column of F); the back substitution in 32-column blocks from the end: one
// warp solves the 32 x 32 diagonal block with shuffles, then all warps fold the
// block into t of the columns to its left.
template <typename T>
__device__ __forceinline__ const T* fac_ptr(const Arenas& A, const NodeDev& nd, int s);
template <> __device__ __forceinline__ const double* fac_ptr<double>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f64 + (int64_t)s * A.f64_stride + nd.f_off;
}
template <> __device__ __forceinline__ const float* fac_ptr<float>(const Arenas& A, const NodeDev& nd, int s) {
  return A.f32 + (int64_t)s * A.f32_stride + nd.f_off;
}

template <typename T>
__device__ __forceinline__ const T* fac_Y(const Arenas& A, const NodeDev& nd, int s) {
  return node_Y<T>(A, nd, s);
}

template <typename T>
__global__ void k_descent(const NodeDev* __restrict__ nodes, const int32_t* __restrict__ maps,
                          const int32_t* __restrict__ list, Arenas A, double* __restrict__ u, int64_t u_stride) {
  const int node = list[blockIdx.x];
  const int s = blockIdx.y;
  const NodeDev nd = nodes[node];
  const int m = nd.m, b = nd.b, nf = nd.nf;
  const T* F = fac_ptr<T>(A, nd, s);
  const int32_t* vid = maps + nd.map_off;
  double* us = u + (int64_t)s * u_stride;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* uB = reinterpret_cast<T*>(smem_raw);   // [b]
  T* t = uB + b;                            // [m]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int i0 = 0; i0 < b; i0 += 4 * blockDim.x) {   // u_B: four gathers per thread in flight
    int v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + q * blockDim.x + threadIdx.x;
      v[q] = i < b ? vid[m + i] : -1;
    }
    double x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) x[q] = v[q] >= 0 ? us[v[q]] : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (v[q] >= 0) uB[i0 + q * blockDim.x + threadIdx.x] = (T)x[q];
  }
  __syncthreads();
  const T* Y = fac_Y<T>(A, nd, s);
  // four columns per warp and pass, their loads in flight together
  for (int c0 = 4 * warp; c0 < m; c0 += 4 * nwarp) {
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
    for (int i = lane; i < b; i += 32) {
      const T ub = uB[i];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c0 + q < m) acc[q] += F[(int64_t)(c0 + q) * nf + m + i] * ub;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (c0 + q < m) t[c0 + q] = Y[c0 + q] - acc[q];
  }
  T* Ld = t + ((m + 3) & ~3);   // [32][33] diagonal block of L_gg, staged per block
  for (int cb = ((m - 1) / 32) * 32; cb >= 0; cb -= 32) {
    const int jb = min(32, m - cb);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * jb; idx += blockDim.x) {
      const int c = idx >> 5, l = idx & 31;
      Ld[c * 33 + l] = (l < jb) ? F[(int64_t)(cb + c) * nf + cb + l] : (T)0;
    }
    __syncthreads();
    if (warp == 0) {
      T x = (lane < jb) ? t[cb + lane] : (T)0;
      for (int r = jb - 1; r >= 0; --r) {
        T ur = __shfl_sync(0xffffffffu, x, r);
        ur = ur / Ld[r * 33 + r];
        if (lane == r) x = ur;
        if (lane < r) x -= Ld[lane * 33 + r] * ur;
      }
      if (lane < jb) t[cb + lane] = x;    // now u_g
    }
    __syncthreads();
    const T ul = (lane < jb) ? t[cb + lane] : (T)0;
    for (int c0 = 4 * warp; c0 < cb; c0 += 4 * nwarp) {   // four columns per pass, loads first
      T acc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        acc[q] = (c0 + q < cb && lane < jb) ? F[(int64_t)(c0 + q) * nf + cb + lane] * ul : (T)0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c0 + q < cb) t[c0 + q] -= acc[q];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += blockDim.x) us[vid[c]] = (double)t[c];
}

template <typename T>
cudaError_t launch_descent(const NodeDev* nodes, const int32_t* maps, const int32_t* list, int nlist, int batch,
                           const Arenas& A, double* u, int64_t u_stride, int max_b, int max_m, cudaStream_t st) {
  if (nlist == 0) return cudaSuccess;
  const size_t smem = ((size_t)max_b + ((max_m + 3) & ~3) + 32 * 33) * sizeof(T);
  k_descent<T><<<dim3(nlist, batch), 256, smem, st>>>(nodes, maps, list, A, u, u_stride);
  return cudaGetLastError();
}
template cudaError_t launch_descent<double>(const NodeDev*, const int32_t*, const int32_t*, int, int, const Arenas&,
                                            double*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_descent<float>(const NodeDev*, const int32_t*, const int32_t*, int, int, const Arenas&,
                                           double*, int64_t, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
__global__ void k_gather_obs(const double* __restrict__ u, int64_t u_stride, const int32_t* __restrict__ obs,
                             int n_obs, double* __restrict__ u_obs) {
  const int s = blockIdx.y;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_obs) u_obs[(int64_t)s * n_obs + k] = u[(int64_t)s * u_stride + obs[k]];
}

cudaError_t launch_gather_obs(const double* u, int64_t u_stride, const int32_t* obs, int n_obs, int batch,
                              double* u_obs, cudaStream_t st) {
  k_gather_obs<<<dim3((n_obs + 255) / 256, batch), 256, 0, st>>>(u, u_stride, obs, n_obs, u_obs);
  return cudaGetLastError();
}

// Likelihood of Sec. 1.2 with Gaussian noise: one CTA per sample, fixed-order
// reduction (each thread strides over k, then a shared-memory tree).
__global__ void k_loglik(const double* __restrict__ u_obs, int n_obs, const double* __restrict__ y,
                         int y_per_sample, double sigma, const int32_t* __restrict__ status,
                         double* __restrict__ loglik) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  const double* us = u_obs + (int64_t)s * n_obs;
  const double* ys = y + (y_per_sample ? (int64_t)s * n_obs : 0);
  double acc = 0.0;
  for (int k = threadIdx.x; k < n_obs; k += blockDim.x) {
    const double r = ys[k] - us[k];
    acc = fma(r, r, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double pi = 3.141592653589793238462643383279502884;
    double ll = -0.5 * red[0] / (sigma * sigma) - 0.5 * n_obs * log(2.0 * pi * sigma * sigma);
    if (status && status[s] != 0) ll = -INFINITY;
    loglik[s] = ll;
  }
}

cudaError_t launch_loglik(const double* u_obs, int n_obs, int batch, const double* y, int y_per_sample, double sigma,
                          const int32_t* status, double* loglik, cudaStream_t st) {
  k_loglik<<<batch, 256, 0, st>>>(u_obs, n_obs, y, y_per_sample, sigma, status, loglik);
  return cudaGetLastError();
}

cudaError_t configure_solve_kernels() {
  const int lim = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_descent<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  if ((e = cudaFuncSetAttribute(k_descent<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim))) return e;
  return cudaSuccess;
}

}  // namespace hdd
