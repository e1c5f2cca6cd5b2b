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
// TwoProduct via FMA (Dekker's product).  exp follows Tang's table-driven method
// (ACM TOMS 15, 1989): q = (16 m + j) ln2/16 + r with |r| <= ln2/32 (ln2/16 as a
// hi/lo pair, the product with the integer formed exactly), e^q = 2^m 2^(j/16) e^r,
// 2^(j/16) from a table of hi/lo pairs and e^r from its Taylor series to degree 6
// (remainder about 2^-51 at |r| = ln2/32), the terms of degree 5 and 6 in FP32 and
// the rest by double-float Horner steps.  Outputs the FP64 kappa (residual), built from the
// hi/lo pair and 2^m by integer operations (the FP64 pipe is the slowest on this
// part), and its FP32 copy (factorisation).
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
__device__ __forceinline__ dflt df_mul_f(dflt a, float b) {   // double-float times an FP32 value
  const float p = a.hi * b;
  const float e = fmaf(a.lo, b, fmaf(a.hi, b, -p));
  return qsum(p, e);
}
// 1/n! for n = 0..4 as hi + lo pairs (the FP32 value nearest to 1/n!, then the
// nearest to the rest); 1/5!, 1/6! in FP32
__constant__ float kInvFact[5][2] = {{1.0f, 0.0f}, {1.0f, 0.0f}, {0.5f, 0.0f},
                                     {0.1666666716337204f, -4.967053879312289e-09f},
                                     {0.0416666679084301f, -1.2417634698280722e-09f}};
constexpr float kInv120 = 0.008333333767950535f, kInv720 = 0.0013888889225199819f;
// 2^(j/16), j = 0..15, as hi + lo pairs (computed to 200 bits, then rounded as above)
__constant__ float kExp2J16[16][2] = {
    {1.0f, 0.0f}, {1.0442737340927124f, 4.8334701574503924e-08f},
    {1.0905077457427979f, -1.3077539939843064e-08f}, {1.1387885808944702f, 5.386222312608879e-08f},
    {1.1892070770263672f, 3.797635272917432e-08f}, {1.2418577671051025f, 4.496838101886169e-08f},
    {1.2968395948410034f, -4.018999533172973e-08f}, {1.3542555570602417f, -1.0123349269974824e-08f},
    {1.4142135381698608f, 2.4203234971764687e-08f}, {1.4768261909484863f, -4.500898853621038e-08f},
    {1.5422108173370361f, 8.070904833346049e-09f}, {1.610490322113037f, 9.836217174097328e-09f},
    {1.6817928552627563f, -2.4755326677450284e-08f}, {1.7562521696090698f, -9.235770370707996e-09f},
    {1.8340080976486206f, -1.1239277952768134e-08f}, {1.9152065515518188f, 9.845328108326612e-09f}};
// ln 2 as hi + lo; 16 / ln 2 rounded to FP32 (only chooses the reduction's integer)
constexpr float kLn2Hi = 0.6931471824645996f, kLn2Lo = -1.9046542121259336e-09f;
constexpr float kSixteenOverLn2 = 23.083120346069336f;

// e^q = 2^m (hi + lo) with hi in [0.97, 2.04)
__device__ __forceinline__ dflt df_exp(dflt q, int* m_out) {
  const float kf = rintf(q.hi * kSixteenOverLn2);
  const float c_hi = kLn2Hi * 0.0625f, c_lo = kLn2Lo * 0.0625f;   // ln2 / 16, exactly scaled
  dflt kl = {kf * c_hi, 0.0f};
  kl.lo = fmaf(kf, c_hi, -kl.hi);          // k ln2_hi / 16 exactly, as hi + lo
  kl.lo = fmaf(kf, c_lo, kl.lo);
  const dflt r = df_add(q, dflt{-kl.hi, -kl.lo});
  const float t = fmaf(r.hi, kInv720, kInv120);               // 1/5! + r/6!
  dflt p = df_add(df_mul_f(r, t), dflt{kInvFact[4][0], kInvFact[4][1]});
#pragma unroll
  for (int n = 3; n >= 0; --n) p = df_add(df_mul(p, r), dflt{kInvFact[n][0], kInvFact[n][1]});
  const int k = (int)kf;
  *m_out = k >> 4;                                           // floor(k / 16)
  const int j = k & 15;
  return df_mul(p, dflt{kExp2J16[j][0], kExp2J16[j][1]});
}

// The double nearest to 2^m (x.hi + x.lo), for x.hi a normal positive FP32 value and
// |x.lo| <= ulp(x.hi) / 2: the 53-bit significand is x.hi's 24 bits shifted up plus x.lo
// in units of the double's last place (rounded to nearest); 0 below the normal range,
// +inf above it.
__device__ __forceinline__ double df_to_double_scaled(dflt x, int m) {
  const uint32_t hb = __float_as_uint(x.hi);
  int e = (int)(hb >> 23) - 127;                             // x.hi = mant 2^(e-23)
  const long long mant = (long long)((hb & 0x7FFFFFu) | 0x800000u);
  const float unit = __int_as_float((127 + 52 - e) << 23);   // 2^(52-e): x.lo in units of 2^(e-52)
  long long M = (mant << 29) + (long long)__float2int_rn(x.lo * unit);
  if (M < (1LL << 52)) {   // x.lo < 0 took x.hi = 2^e below it
    M <<= 1;
    --e;
  }
  const int ef = e + m + 1023;
  if (ef >= 2047) return __longlong_as_double(0x7FF0000000000000LL);
  if (ef <= 0) return 0.0;
  return __longlong_as_double(((long long)ef << 52) | (M & ((1LL << 52) - 1)));
}

// 2^m x for a normal positive FP32 x: the exponent field moved by m, or ldexpf
// where the result leaves the normal range
__device__ __forceinline__ float scale_pow2(float x, int m) {
  const int e = (int)(__float_as_uint(x) >> 23) + m;
  return (e >= 1 && e <= 254) ? __int_as_float((int)__float_as_uint(x) + (m << 23)) : ldexpf(x, m);
}
}  // namespace

// CTA = 128 triangles x 8 samples; the sample groups of one triangle block are
// consecutive CTAs (blockIdx.x = triangle block x groups + group), so the block's
// Phi rows are read from HBM once and from L2 by the other groups.  Z is staged
// with the samples innermost: a column's eight samples are two 16-byte loads.
__global__ void k_kappa_df(const float* __restrict__ phi_hi, const float* __restrict__ phi_lo,
                           const double* __restrict__ Z, int n_t, int n_z, int batch, double* __restrict__ kappa,
                           float* __restrict__ kappa32, int64_t kap_stride) {
  __shared__ float ph[kKapK][kKapT + 1], pl[kKapK][kKapT + 1];
  __shared__ __align__(16) float zh[kKapK][kKapS], zl[kKapK][kKapS];
  const int n_groups = (batch + kKapS - 1) / kKapS;
  const int t0 = (blockIdx.x / n_groups) * kKapT, s0 = (blockIdx.x % n_groups) * kKapS;
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
      zh[kk][ss] = h;
      zl[kk][ss] = (float)(z - (double)h);
    }
    __syncthreads();
    for (int kk = 0; kk < kc; ++kk) {
      const float a = ph[kk][threadIdx.x], b = pl[kk][threadIdx.x];
      float zq[kKapS], zr[kKapS];
#pragma unroll
      for (int q4 = 0; q4 < kKapS; q4 += 4) {
        const float4 u = *reinterpret_cast<const float4*>(&zh[kk][q4]);
        const float4 v = *reinterpret_cast<const float4*>(&zl[kk][q4]);
        zq[q4] = u.x; zq[q4 + 1] = u.y; zq[q4 + 2] = u.z; zq[q4 + 3] = u.w;
        zr[q4] = v.x; zr[q4 + 1] = v.y; zr[q4 + 2] = v.z; zr[q4 + 3] = v.w;
      }
#pragma unroll
      for (int q = 0; q < kKapS; ++q) {
        const float p = a * zq[q];
        float e = fmaf(a, zq[q], -p);
        e = fmaf(a, zr[q], fmaf(b, zq[q], e));
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
      int m;
      const dflt ex = df_exp(qsum(ah[q], al[q]), &m);
      kappa[(int64_t)(s0 + q) * kap_stride + t] = df_to_double_scaled(ex, m);
      kappa32[(int64_t)(s0 + q) * kap_stride + t] = scale_pow2(ex.hi, m);
    }
  }
}

cudaError_t launch_kappa_df(const float* phi_hi, const float* phi_lo, const double* Z, int n_t, int n_z, int batch,
                            double* kappa, float* kappa32, int64_t kap_stride, cudaStream_t st) {
  const int64_t blocks = (int64_t)((n_t + kKapT - 1) / kKapT) * ((batch + kKapS - 1) / kKapS);
  if (blocks > INT32_MAX) return cudaErrorInvalidConfiguration;
  k_kappa_df<<<(unsigned)blocks, kKapT, 0, st>>>(phi_hi, phi_lo, Z, n_t, n_z, batch, kappa, kappa32, kap_stride);
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
