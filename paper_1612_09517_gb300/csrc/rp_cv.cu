// Learned control variate for the stochastic trace estimate (Eqs. 18, 23).
//
// A multilayer perceptron g(Omega, B) (SiLU hidden layers, linear output,
// BF16 weights, FP32 activations and accumulation) is trained on per-sample
// yields phi_S(Omega_s, B) produced by rp_yields, then used as a control
// variate: Phi_cv = mean(phi - beta (g - mu)) with mu = E_Omega[g] from many
// fresh directions (inference only) and beta = cov(phi, g) / var(g).  Any g
// fixed before the estimation samples are drawn leaves the estimate
// unbiased; a good g lowers its variance.
//
// Features of a sample (regenerated on the device from the same Philox map as
// the initial states): per nucleus k in input order the direction
// n(Omega_k) = (sin t cos p, sin t sin p, cos t) (Eq. 16), then B / B_scale.
// Parameters are one flat FP32 vector W_0, b_0, W_1, b_1, ... (W_l row-major
// (out, in)); the forward pass uses the BF16-rounded copy of the weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "../../include/rp.h"
#include "rp_kernels.cuh"
#include "rp_plan.h"

struct rp_system {
  rp::HostSystem hs;
};

namespace rp {
void set_last_error(const std::string& msg);
void* device_alloc(size_t bytes, cudaStream_t st);
void device_free(void* p, cudaStream_t st);
rp_status device_check();
}  // namespace rp

struct rp_cv {
  int n_nuc = 0, d_in = 0, hidden = 0, layers = 0;
  double B_scale = 10.0;
  rp_cv_options opt{};
  long long n_params = 0;
  std::vector<long long> w_off, b_off;  // per layer, in the flat vector
  std::vector<int> rows, cols;          // per layer (out, in)
  float* master = nullptr;              // FP32 parameters
  float* m1 = nullptr;                  // Adam first moments
  float* m2 = nullptr;                  // Adam second moments
  __nv_bfloat16* wbf = nullptr;         // BF16 copy of the weights (same offsets)
  float* nuc = nullptr;                 // per nucleus I_k A_k / B_hyp (9) and radical
  long long adam_t = 0;
  cudaStream_t st = nullptr;
};

namespace {

rp_status cfail(rp_status s, const std::string& m) {
  rp::set_last_error(m);
  return s;
}

struct CvFail {
  rp_status st;
  std::string msg;
};

void cck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw CvFail{e == cudaErrorMemoryAllocation ? RP_ENOMEM : RP_ECUDA,
                 std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

template <typename T>
T* dalloc(size_t n, cudaStream_t st) {
  void* p = rp::device_alloc(std::max<size_t>(n, 1) * sizeof(T), st);
  if (!p) throw CvFail{RP_ENOMEM, "device allocation failed"};
  return static_cast<T*>(p);
}

// Scratch released when the scope ends.
struct Scratch {
  cudaStream_t st;
  std::vector<void*> p;
  template <typename T>
  T* get(size_t n) {
    T* q = dalloc<T>(n, st);
    p.push_back(q);
    return q;
  }
  ~Scratch() {
    for (auto it = p.rbegin(); it != p.rend(); ++it) rp::device_free(*it, st);
  }
};

inline unsigned g1(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ void philox(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
    const uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  return ((double)(hi >> 5) * 67108864.0 + (double)(lo >> 6)) * (1.0 / 9007199254740992.0);
}

// Features of sample samples[i] (or sample0 + i) at field B_i (or B_one), one
// thread per sample:
//   x[3k .. 3k+2] = n(Omega_k), k in input order (Eq. 16 direction of the draw);
//   x[3N .. 3N+5] = b_1, b_2 with b_r = sum_{k on r} (I_k A_k / B_hyp,r) n(Omega_k);
//   x[3N+6 .. 3N+8] = |b_1|, |b_2|, b_1 . b_2;   x[3N+9] = B / B_scale.
// nuc[10 k .. 10 k + 8] = I_k A_k / B_hyp,r(k) row-major, nuc[10 k + 9] = radical.
__global__ void k_features(int n, int n_nuc, const float* __restrict__ nuc,
                           const double* __restrict__ B, double B_one,
                           const long long* __restrict__ samples, long long sample0, uint64_t seed,
                           uint32_t pair, double inv_scale, float* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int d_in = 3 * n_nuc + 10;
  float* xi = x + (size_t)i * d_in;
  const unsigned long long s = (unsigned long long)(samples ? samples[i] : sample0 + i);
  float b[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  for (int k = 0; k < n_nuc; ++k) {
    uint32_t c[4] = {(uint32_t)k, (uint32_t)(s & 0xFFFFFFFFull), (uint32_t)(s >> 32), pair};
    philox(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
    const double ct = 1.0 - 2.0 * u1;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sp, cp;
    sincospi(2.0 * u2, &sp, &cp);
    const float v[3] = {(float)(st * cp), (float)(st * sp), (float)ct};
    xi[3 * k] = v[0];
    xi[3 * k + 1] = v[1];
    xi[3 * k + 2] = v[2];
    const float* Mk = nuc + 10 * k;
    const int r = (int)Mk[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) b[r][a] += Mk[3 * a] * v[0] + Mk[3 * a + 1] * v[1] + Mk[3 * a + 2] * v[2];
  }
  float* t = xi + 3 * n_nuc;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    t[a] = b[0][a];
    t[3 + a] = b[1][a];
  }
  t[6] = sqrtf(b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2]);
  t[7] = sqrtf(b[1][0] * b[1][0] + b[1][1] * b[1][1] + b[1][2] * b[1][2]);
  t[8] = b[0][0] * b[1][0] + b[0][1] * b[1][1] + b[0][2] * b[1][2];
  t[9] = (float)((B ? B[i] : B_one) * inv_scale);
}

__device__ __forceinline__ float ld(const float* p, long long i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

// C[m][n] (+)= sum_k A(m, k) B(k, n), A(m, k) = A[m a_m + k a_k], B(k, n) = B[k b_k + n b_n],
// FP32 accumulation; 64 x 64 tiles, k-chunks of 16, 256 threads x (4 x 4) outputs.
constexpr int kT = 64, kK = 16;

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const TA* __restrict__ A,
                                              long long a_m, long long a_k,
                                              const TB* __restrict__ B, long long b_k,
                                              long long b_n, float* __restrict__ C, long long c_m,
                                              int accumulate) {
  __shared__ float As[kK][kT + 4];
  __shared__ float Bs[kK][kT + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * kT, n0 = blockIdx.x * kT;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;  // 0..1023
      const int mm = e / kK, kk = e % kK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? ld(A, (long long)gm * a_m + (long long)gk * a_k) : 0.f;
      const int nn = e / kK;
      const int gn = n0 + nn;
      Bs[kk][nn] = (gn < N && gk < K) ? ld(B, (long long)gk * b_k + (long long)gn * b_n) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float* c = C + (long long)gm * c_m + gn;
      *c = accumulate ? (*c + acc[i][j]) : acc[i][j];
    }
  }
}

// z = y + b (row broadcast); a = silu(z) when act, else a = z.
__global__ void k_bias_act(int n, int out, const float* __restrict__ b, float* __restrict__ z,
                           float* __restrict__ a, int act) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * out) return;
  const float v = z[t] + b[t % out];
  z[t] = v;
  a[t] = act ? v / (1.f + __expf(-v)) : v;
}

// dz = dh * silu'(z), silu'(z) = s (1 + z (1 - s)), s = 1 / (1 + e^-z).
__global__ void k_silu_back(long long n, const float* __restrict__ z, float* __restrict__ dh) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float v = z[t];
  const float s = 1.f / (1.f + __expf(-v));
  dh[t] *= s * (1.f + v * (1.f - s));
}

// db[o] = sum_i dz[i][o]
__global__ void k_bias_grad(int n, int out, const float* __restrict__ dz, float* __restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= out) return;
  float s = 0.f;
  for (int i = 0; i < n; ++i) s += dz[(size_t)i * out + o];
  db[o] = s;
}

template <int NT>
__device__ double bsum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// r = g - y; dz = r / n (gradient of the batch mean); loss += sum r^2 / (2 n_total)
__global__ void __launch_bounds__(256) k_mse(int n, double n_total, const float* __restrict__ g,
                                             const float* __restrict__ y, float* __restrict__ dz,
                                             double* __restrict__ loss) {
  __shared__ double sh[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (i < n) {
    const float r = g[i] - y[i];
    dz[i] = (float)((double)r / (double)n);
    v = 0.5 * (double)r * (double)r / n_total;
  }
  const double t = bsum<256>(v, sh);
  if (threadIdx.x == 0) atomicAdd(loss, t);
}

// Adam (Kingma and Ba 2015) with decoupled weight decay on the weights; keeps
// the BF16 copy of each weight in step.
__global__ void k_adam(long long n, float* __restrict__ w, float* __restrict__ m1,
                       float* __restrict__ m2, const float* __restrict__ g,
                       __nv_bfloat16* __restrict__ wbf, const unsigned char* __restrict__ is_w,
                       float lr, float b1, float b2, float c1, float c2, float eps, float wd) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  float wi = w[i];
  if (is_w[i]) wi -= lr * wd * wi;
  wi -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  w[i] = wi;
  wbf[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(long long n, const float* __restrict__ w, __nv_bfloat16* __restrict__ o) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = __float2bfloat16(w[i]);
}

__global__ void k_gather(int n, int d, const int* __restrict__ idx, const float* __restrict__ src,
                         float* __restrict__ dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * d) return;
  const int i = (int)(t / d), j = (int)(t % d);
  dst[t] = src[(size_t)idx[i] * d + j];
}

// acc[0] += sum g, acc[1] += sum g^2 (FP64)
__global__ void __launch_bounds__(256) k_moments(int n, const float* __restrict__ g,
                                                 double* __restrict__ acc) {
  __shared__ double sh[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double v = i < n ? (double)g[i] : 0.0;
  const double s1 = bsum<256>(v, sh);
  __syncthreads();
  const double s2 = bsum<256>(v * v, sh);
  if (threadIdx.x == 0) {
    atomicAdd(acc, s1);
    atomicAdd(acc + 1, s2);
  }
}

// Control-variate estimate of one field per block over its samples
// [off, off + cnt): phi (stride 3 in ps) and g; mu and var(mu) per field.
// out[f] = {Phi_cv, SE_cv, Phi_plain, SE_plain, beta}
__global__ void __launch_bounds__(256) k_cv_stats(const double* __restrict__ ps,
                                                  const float* __restrict__ g,
                                                  const long long* __restrict__ off,
                                                  const long long* __restrict__ cnt,
                                                  const double* __restrict__ mu,
                                                  const double* __restrict__ var_mu,
                                                  double* __restrict__ out) {
  __shared__ double sh[256];
  const int f = blockIdx.x;
  const long long o = off[f], M = cnt[f];
  double sp = 0, sg = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    sp += ps[(o + i) * 3];
    sg += (double)g[o + i];
  }
  const double Md = M > 0 ? (double)M : 1.0;
  const double mp = bsum<256>(sp, sh) / Md;
  __syncthreads();
  const double mg = bsum<256>(sg, sh) / Md;
  __syncthreads();
  double cpp = 0, cpg = 0, cgg = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    const double dp = ps[(o + i) * 3] - mp, dg = (double)g[o + i] - mg;
    cpp += dp * dp;
    cpg += dp * dg;
    cgg += dg * dg;
  }
  const double Spp = bsum<256>(cpp, sh);
  __syncthreads();
  const double Spg = bsum<256>(cpg, sh);
  __syncthreads();
  const double Sgg = bsum<256>(cgg, sh);
  if (threadIdx.x == 0) {
    const double den = M > 1 ? (double)(M - 1) : 1.0;
    const double beta = Sgg > 0 ? Spg / Sgg : 0.0;
    // var(phi - beta g) with the sample covariances
    const double vres = fmax(0.0, (Spp - 2.0 * beta * Spg + beta * beta * Sgg) / den);
    out[5 * f + 0] = mp - beta * (mg - mu[f]);
    out[5 * f + 1] = sqrt(vres / Md + beta * beta * var_mu[f]);
    out[5 * f + 2] = mp;
    out[5 * f + 3] = sqrt(Spp / den / Md);
    out[5 * f + 4] = beta;
  }
}

// ------------------------------------------------------------- host side

void gemm_ff(int M, int N, int K, const float* A, long long a_m, long long a_k, const float* B,
             long long b_k, long long b_n, float* C, long long c_m, int accumulate, cudaStream_t st) {
  dim3 grid(g1(N, kT), g1(M, kT));
  k_gemm<float, float><<<grid, 256, 0, st>>>(M, N, K, A, a_m, a_k, B, b_k, b_n, C, c_m, accumulate);
  cck(cudaGetLastError(), "gemm");
}
void gemm_fb(int M, int N, int K, const float* A, long long a_m, long long a_k,
             const __nv_bfloat16* B, long long b_k, long long b_n, float* C, long long c_m,
             int accumulate, cudaStream_t st) {
  dim3 grid(g1(N, kT), g1(M, kT));
  k_gemm<float, __nv_bfloat16><<<grid, 256, 0, st>>>(M, N, K, A, a_m, a_k, B, b_k, b_n, C, c_m,
                                                     accumulate);
  cck(cudaGetLastError(), "gemm");
}

// Activations of a batch: z[l] and a[l] per layer (input x), and the
// backward buffers dh[l] (n x in of layer l, l >= 1).
struct Acts {
  std::vector<float*> z, a, dh;
};

Acts make_acts(rp_cv* cv, int n, Scratch& sc) {
  Acts A;
  for (int l = 0; l <= cv->layers; ++l) {
    A.z.push_back(sc.get<float>((size_t)n * cv->rows[l]));
    A.a.push_back(sc.get<float>((size_t)n * cv->rows[l]));
    A.dh.push_back(l > 0 ? sc.get<float>((size_t)n * cv->cols[l]) : nullptr);
  }
  return A;
}

// g = A.a[layers] (n x 1)
void forward(rp_cv* cv, int n, const float* x, Acts& A, cudaStream_t st) {
  const float* h = x;
  for (int l = 0; l <= cv->layers; ++l) {
    const int out = cv->rows[l], in = cv->cols[l];
    // z[i][o] = sum_j h[i][j] W[o][j]
    gemm_fb(n, out, in, h, in, 1, cv->wbf + cv->w_off[l], 1, in, A.z[l], out, 0, st);
    k_bias_act<<<g1((long long)n * out, 256), 256, 0, st>>>(n, out, cv->master + cv->b_off[l],
                                                            A.z[l], A.a[l], l < cv->layers);
    cck(cudaGetLastError(), "bias/activation");
    h = A.a[l];
  }
}

// grad = d loss / d params for dz_L given (n x 1), using the BF16 weights.
void backward(rp_cv* cv, int n, const float* x, Acts& A, float* dz_last, float* grad,
              cudaStream_t st) {
  float* dz = dz_last;
  for (int l = cv->layers; l >= 0; --l) {
    const int out = cv->rows[l], in = cv->cols[l];
    const float* h = l > 0 ? A.a[l - 1] : x;
    // dW[o][j] = sum_i dz[i][o] h[i][j]
    gemm_ff(out, in, n, dz, 1, out, h, in, 1, grad + cv->w_off[l], in, 0, st);
    k_bias_grad<<<g1(out, 128), 128, 0, st>>>(n, out, dz, grad + cv->b_off[l]);
    cck(cudaGetLastError(), "bias grad");
    if (l > 0) {
      // dh[i][j] = sum_o dz[i][o] W[o][j]
      float* dh = A.dh[l];
      gemm_fb(n, in, out, dz, out, 1, cv->wbf + cv->w_off[l], in, 1, dh, in, 0, st);
      k_silu_back<<<g1((long long)n * in, 256), 256, 0, st>>>((long long)n * in, A.z[l - 1], dh);
      cck(cudaGetLastError(), "silu backward");
      dz = dh;
    }
  }
}

void features_dev(rp_cv* cv, int n, const double* d_B, double B_one, const long long* d_samples,
                  long long sample0, uint64_t seed, uint32_t pair, float* x, cudaStream_t st) {
  k_features<<<g1(n, 128), 128, 0, st>>>(n, cv->n_nuc, cv->nuc, d_B, B_one, d_samples, sample0,
                                         seed, pair, 1.0 / cv->B_scale, x);
  cck(cudaGetLastError(), "features");
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

void rp_cv_default_options(rp_cv_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hidden = 256;
  o->layers = 3;
  o->epochs = 200;
  o->batch = 256;
  o->lr = 1e-3;
  o->weight_decay = 1e-4;
  o->B_scale = 10.0;
  o->init_seed = 1;
}

rp_status rp_cv_create(const rp_system* sys, const rp_cv_options* opt, rp_cv** out) {
  rp::set_last_error("");
  if (!sys || !out) return cfail(RP_EINVAL, "NULL argument");
  *out = nullptr;
  rp_cv_options o;
  if (opt) o = *opt;
  else rp_cv_default_options(&o);
  if (o.hidden < 1 || o.hidden > 4096 || o.layers < 1 || o.layers > 8)
    return cfail(RP_EINVAL, "hidden must be in [1, 4096] and layers in [1, 8]");
  if (!(o.B_scale > 0.0)) return cfail(RP_EINVAL, "B_scale must be positive");
  rp_status ds = rp::device_check();
  if (ds != RP_OK) return ds;
  rp_cv* cv = new rp_cv;
  cv->opt = o;
  cv->st = (cudaStream_t)o.stream;
  cv->n_nuc = sys->hs.n_nuc;
  cv->d_in = 3 * cv->n_nuc + 10;
  cv->hidden = o.hidden;
  cv->layers = o.layers;
  cv->B_scale = o.B_scale;
  long long off = 0;
  for (int l = 0; l <= o.layers; ++l) {
    const int in = l == 0 ? cv->d_in : o.hidden;
    const int outd = l == o.layers ? 1 : o.hidden;
    cv->rows.push_back(outd);
    cv->cols.push_back(in);
    cv->w_off.push_back(off);
    off += (long long)outd * in;
    cv->b_off.push_back(off);
    off += outd;
  }
  cv->n_params = off;
  // He-style uniform initialisation (scale sqrt(3 / fan_in) for SiLU layers), zero biases
  std::vector<float> p(off, 0.f);
  std::mt19937_64 rng(o.init_seed);
  for (int l = 0; l <= o.layers; ++l) {
    const double a = std::sqrt((l < o.layers ? 6.0 : 3.0) / cv->cols[l]);
    std::uniform_real_distribution<double> U(-a, a);
    for (long long i = 0; i < (long long)cv->rows[l] * cv->cols[l]; ++i) p[cv->w_off[l] + i] = (float)U(rng);
  }
  // I_k A_k / B_hyp,r for the hyperfine-field features (B_hyp of Eq. 21 with
  // a_k^2 -> |A_k|_F^2 / 3 for anisotropic tensors)
  const rp::HostSystem& hs = sys->hs;
  std::vector<float> nuc(10 * std::max(cv->n_nuc, 1), 0.f);
  {
    double bh2[2] = {0.0, 0.0};
    for (int k = 0; k < hs.n_nuc; ++k) {
      const double I = 0.5 * hs.two_I[k];
      double f2 = 0.0;
      for (int q = 0; q < 9; ++q) f2 += hs.A[9 * k + q] * hs.A[9 * k + q];
      bh2[hs.radical[k]] += f2 / 3.0 * I * (I + 1.0);
    }
    for (int k = 0; k < hs.n_nuc; ++k) {
      const int r = hs.radical[k];
      const double I = 0.5 * hs.two_I[k];
      const double sc = bh2[r] > 0.0 ? I / std::sqrt(bh2[r]) : 0.0;
      for (int q = 0; q < 9; ++q) nuc[10 * k + q] = (float)(sc * hs.A[9 * k + q]);
      nuc[10 * k + 9] = (float)r;
    }
  }
  try {
    cv->nuc = dalloc<float>(nuc.size(), cv->st);
    cck(cudaMemcpyAsync(cv->nuc, nuc.data(), nuc.size() * sizeof(float), cudaMemcpyHostToDevice, cv->st), "h2d");
    cv->master = dalloc<float>(off, cv->st);
    cv->m1 = dalloc<float>(off, cv->st);
    cv->m2 = dalloc<float>(off, cv->st);
    cv->wbf = dalloc<__nv_bfloat16>(off, cv->st);
    cck(cudaMemcpyAsync(cv->master, p.data(), off * sizeof(float), cudaMemcpyHostToDevice, cv->st), "h2d");
    cck(cudaMemsetAsync(cv->m1, 0, off * sizeof(float), cv->st), "memset");
    cck(cudaMemsetAsync(cv->m2, 0, off * sizeof(float), cv->st), "memset");
    k_to_bf16<<<g1(off, 256), 256, 0, cv->st>>>(off, cv->master, cv->wbf);
    cck(cudaGetLastError(), "bf16");
    cck(cudaStreamSynchronize(cv->st), "create");
  } catch (const CvFail& e) {
    rp_cv_destroy(cv);
    return cfail(e.st, e.msg);
  }
  *out = cv;
  return RP_OK;
}

void rp_cv_destroy(rp_cv* cv) {
  if (!cv) return;
  rp::device_free(cv->master, cv->st);
  rp::device_free(cv->m1, cv->st);
  rp::device_free(cv->m2, cv->st);
  rp::device_free(cv->wbf, cv->st);
  rp::device_free(cv->nuc, cv->st);
  cudaStreamSynchronize(cv->st);
  delete cv;
}

rp_status rp_cv_params(rp_cv* cv, float* get, const float* set, long long* count) {
  rp::set_last_error("");
  if (!cv) return cfail(RP_EINVAL, "NULL model");
  if (count) *count = cv->n_params;
  try {
    if (set) {
      cck(cudaMemcpyAsync(cv->master, set, cv->n_params * sizeof(float), cudaMemcpyHostToDevice, cv->st), "h2d");
      k_to_bf16<<<g1(cv->n_params, 256), 256, 0, cv->st>>>(cv->n_params, cv->master, cv->wbf);
      cck(cudaGetLastError(), "bf16");
    }
    if (get)
      cck(cudaMemcpyAsync(get, cv->master, cv->n_params * sizeof(float), cudaMemcpyDeviceToHost, cv->st), "d2h");
    cck(cudaStreamSynchronize(cv->st), "params");
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_cv_loss_grad(rp_cv* cv, int n, const float* x, const float* y, double* loss,
                          float* grad) {
  rp::set_last_error("");
  if (!cv || n < 1 || !x || !y) return cfail(RP_EINVAL, "bad arguments");
  try {
    Scratch sc{cv->st};
    float* dx = sc.get<float>((size_t)n * cv->d_in);
    float* dy = sc.get<float>(n);
    float* dzl = sc.get<float>(n);
    float* dg = sc.get<float>(cv->n_params);
    double* dl = sc.get<double>(1);
    cck(cudaMemcpyAsync(dx, x, (size_t)n * cv->d_in * sizeof(float), cudaMemcpyHostToDevice, cv->st), "h2d");
    cck(cudaMemcpyAsync(dy, y, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, cv->st), "h2d");
    cck(cudaMemsetAsync(dl, 0, sizeof(double), cv->st), "memset");
    Acts A = make_acts(cv, n, sc);
    forward(cv, n, dx, A, cv->st);
    k_mse<<<g1(n, 256), 256, 0, cv->st>>>(n, (double)n, A.a[cv->layers], dy, dzl, dl);
    cck(cudaGetLastError(), "mse");
    backward(cv, n, dx, A, dzl, dg, cv->st);
    if (loss) cck(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, cv->st), "d2h");
    if (grad) cck(cudaMemcpyAsync(grad, dg, cv->n_params * sizeof(float), cudaMemcpyDeviceToHost, cv->st), "d2h");
    cck(cudaStreamSynchronize(cv->st), "loss/grad");
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_cv_train(rp_cv* cv, int n, const double* B, const long long* samples, uint64_t seed,
                      uint32_t pair_id, const double* phi, double* loss_per_epoch) {
  rp::set_last_error("");
  if (!cv || n < 2 || !B || !samples || !phi) return cfail(RP_EINVAL, "bad arguments");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(B[i]) || !std::isfinite(phi[i]) || samples[i] < 0)
      return cfail(RP_EINVAL, "non-finite training data or negative sample index");
  const rp_cv_options& o = cv->opt;
  cudaStream_t st = cv->st;
  // targets: per-field standardised phi (the control variate needs only the
  // within-field variation; the field enters through the last feature)
  std::vector<float> y(n);
  {
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return B[a] < B[b]; });
    for (int i0 = 0; i0 < n;) {
      int i1 = i0;
      while (i1 < n && B[idx[i1]] == B[idx[i0]]) ++i1;
      double m = 0, v = 0;
      for (int i = i0; i < i1; ++i) m += phi[idx[i]];
      m /= (i1 - i0);
      for (int i = i0; i < i1; ++i) v += (phi[idx[i]] - m) * (phi[idx[i]] - m);
      const double sd = (i1 - i0 > 1 && v > 0) ? std::sqrt(v / (i1 - i0 - 1)) : 1.0;
      for (int i = i0; i < i1; ++i) y[idx[i]] = (float)((phi[idx[i]] - m) / sd);
      i0 = i1;
    }
  }
  try {
    Scratch sc{st};
    double* dB = sc.get<double>(n);
    long long* ds = sc.get<long long>(n);
    float* X = sc.get<float>((size_t)n * cv->d_in);
    float* Y = sc.get<float>(n);
    cck(cudaMemcpyAsync(dB, B, n * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
    cck(cudaMemcpyAsync(ds, samples, n * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    cck(cudaMemcpyAsync(Y, y.data(), n * sizeof(float), cudaMemcpyHostToDevice, st), "h2d");
    features_dev(cv, n, dB, 0.0, ds, 0, seed, pair_id, X, st);
    const int bs = std::min(std::max(o.batch, 1), n);
    float* xb = sc.get<float>((size_t)bs * cv->d_in);
    float* yb = sc.get<float>(bs);
    float* dzl = sc.get<float>(bs);
    float* grad = sc.get<float>(cv->n_params);
    double* dloss = sc.get<double>(std::max(o.epochs, 1));
    int* perm_d = sc.get<int>(n);
    unsigned char* is_w = sc.get<unsigned char>(cv->n_params);
    {
      std::vector<unsigned char> w(cv->n_params, 0);
      for (int l = 0; l <= cv->layers; ++l)
        for (long long i = 0; i < (long long)cv->rows[l] * cv->cols[l]; ++i) w[cv->w_off[l] + i] = 1;
      cck(cudaMemcpyAsync(is_w, w.data(), w.size(), cudaMemcpyHostToDevice, st), "h2d");
      cck(cudaStreamSynchronize(st), "h2d");
    }
    cck(cudaMemsetAsync(dloss, 0, std::max(o.epochs, 1) * sizeof(double), st), "memset");
    Acts A = make_acts(cv, bs, sc);
    std::mt19937_64 rng(o.init_seed ^ 0x5bd1e995ull);
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < o.epochs; ++ep) {
      std::shuffle(perm.begin(), perm.end(), rng);
      cck(cudaMemcpyAsync(perm_d, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st), "h2d");
      cck(cudaStreamSynchronize(st), "perm");
      for (int i0 = 0; i0 + bs <= n; i0 += bs) {
        k_gather<<<g1((long long)bs * cv->d_in, 256), 256, 0, st>>>(bs, cv->d_in, perm_d + i0, X, xb);
        k_gather<<<g1(bs, 256), 256, 0, st>>>(bs, 1, perm_d + i0, Y, yb);
        forward(cv, bs, xb, A, st);
        k_mse<<<g1(bs, 256), 256, 0, st>>>(bs, (double)bs * (n / bs), A.a[cv->layers], yb, dzl,
                                           dloss + ep);
        cck(cudaGetLastError(), "mse");
        backward(cv, bs, xb, A, dzl, grad, st);
        cv->adam_t++;
        const float c1 = 1.f - std::pow(b1, (float)cv->adam_t), c2 = 1.f - std::pow(b2, (float)cv->adam_t);
        k_adam<<<g1(cv->n_params, 256), 256, 0, st>>>(cv->n_params, cv->master, cv->m1, cv->m2,
                                                      grad, cv->wbf, is_w, (float)o.lr, b1, b2, c1,
                                                      c2, 1e-8f, (float)o.weight_decay);
        cck(cudaGetLastError(), "adam");
      }
    }
    if (loss_per_epoch)
      cck(cudaMemcpyAsync(loss_per_epoch, dloss, o.epochs * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    cck(cudaStreamSynchronize(st), "train");
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_cv_eval(rp_cv* cv, int n, const double* B, const long long* samples, uint64_t seed,
                     uint32_t pair_id, double* g) {
  rp::set_last_error("");
  if (!cv || n < 0 || (n > 0 && (!B || !samples || !g))) return cfail(RP_EINVAL, "bad arguments");
  if (n == 0) return RP_OK;
  cudaStream_t st = cv->st;
  try {
    Scratch sc{st};
    const int chunk = 65536;
    double* dB = sc.get<double>(std::min(n, chunk));
    long long* ds = sc.get<long long>(std::min(n, chunk));
    float* X = sc.get<float>((size_t)std::min(n, chunk) * cv->d_in);
    Acts A = make_acts(cv, std::min(n, chunk), sc);
    std::vector<float> gf(std::min(n, chunk));
    for (int i0 = 0; i0 < n; i0 += chunk) {
      const int m = std::min(chunk, n - i0);
      cck(cudaMemcpyAsync(dB, B + i0, m * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
      cck(cudaMemcpyAsync(ds, samples + i0, m * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
      features_dev(cv, m, dB, 0.0, ds, 0, seed, pair_id, X, st);
      forward(cv, m, X, A, st);
      cck(cudaMemcpyAsync(gf.data(), A.a[cv->layers], m * sizeof(float), cudaMemcpyDeviceToHost, st), "d2h");
      cck(cudaStreamSynchronize(st), "eval");
      for (int i = 0; i < m; ++i) g[i0 + i] = gf[i];
    }
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_cv_mean(rp_cv* cv, int n_fields, const double* B, long long n_mc, uint64_t seed,
                     uint32_t pair_id, double* mu, double* var_mu) {
  rp::set_last_error("");
  if (!cv || n_fields < 0 || (n_fields > 0 && (!B || !mu)) || n_mc < 2)
    return cfail(RP_EINVAL, "bad arguments");
  if (n_fields == 0) return RP_OK;
  cudaStream_t st = cv->st;
  try {
    Scratch sc{st};
    const int chunk = 65536;
    float* X = sc.get<float>((size_t)chunk * cv->d_in);
    Acts A = make_acts(cv, chunk, sc);
    double* acc = sc.get<double>(2 * (size_t)n_fields);
    cck(cudaMemsetAsync(acc, 0, 2 * n_fields * sizeof(double), st), "memset");
    for (int f = 0; f < n_fields; ++f)
      for (long long s0 = 0; s0 < n_mc; s0 += chunk) {
        const int m = (int)std::min<long long>(chunk, n_mc - s0);
        features_dev(cv, m, nullptr, B[f], nullptr, s0, seed, pair_id, X, st);
        forward(cv, m, X, A, st);
        k_moments<<<g1(m, 256), 256, 0, st>>>(m, A.a[cv->layers], acc + 2 * f);
        cck(cudaGetLastError(), "moments");
      }
    std::vector<double> h(2 * (size_t)n_fields);
    cck(cudaMemcpyAsync(h.data(), acc, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    cck(cudaStreamSynchronize(st), "mean");
    for (int f = 0; f < n_fields; ++f) {
      const double m = h[2 * f] / (double)n_mc;
      const double v = std::max(0.0, (h[2 * f + 1] / (double)n_mc - m * m)) * n_mc / (n_mc - 1.0);
      mu[f] = m;
      if (var_mu) var_mu[f] = v / (double)n_mc;
    }
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_cv_estimate(rp_cv* cv, int n_fields, const long long* offsets, const long long* counts,
                         const double* per_sample, const double* g, const double* mu,
                         const double* var_mu, double* out) {
  rp::set_last_error("");
  if (!cv || n_fields < 0 || (n_fields > 0 && (!offsets || !counts || !per_sample || !g || !mu || !var_mu || !out)))
    return cfail(RP_EINVAL, "bad arguments");
  if (n_fields == 0) return RP_OK;
  long long tot = 0;
  for (int f = 0; f < n_fields; ++f) {
    if (counts[f] < 2 || offsets[f] < 0) return cfail(RP_EINVAL, "each field needs >= 2 samples");
    tot = std::max(tot, offsets[f] + counts[f]);
  }
  cudaStream_t st = cv->st;
  try {
    Scratch sc{st};
    double* dps = sc.get<double>((size_t)tot * 3);
    float* dg = sc.get<float>(tot);
    long long* doc = sc.get<long long>(2 * (size_t)n_fields);
    double* dmu = sc.get<double>(2 * (size_t)n_fields);
    double* dout = sc.get<double>(5 * (size_t)n_fields);
    std::vector<float> gf(tot);
    for (long long i = 0; i < tot; ++i) gf[i] = (float)g[i];
    std::vector<long long> oc(2 * (size_t)n_fields);
    std::vector<double> mv(2 * (size_t)n_fields);
    for (int f = 0; f < n_fields; ++f) {
      oc[f] = offsets[f];
      oc[n_fields + f] = counts[f];
      mv[f] = mu[f];
      mv[n_fields + f] = var_mu[f];
    }
    cck(cudaMemcpyAsync(dps, per_sample, (size_t)tot * 3 * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
    cck(cudaMemcpyAsync(dg, gf.data(), tot * sizeof(float), cudaMemcpyHostToDevice, st), "h2d");
    cck(cudaMemcpyAsync(doc, oc.data(), oc.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    cck(cudaMemcpyAsync(dmu, mv.data(), mv.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
    k_cv_stats<<<n_fields, 256, 0, st>>>(dps, dg, doc, doc + n_fields, dmu, dmu + n_fields, dout);
    cck(cudaGetLastError(), "cv stats");
    cck(cudaMemcpyAsync(out, dout, 5 * (size_t)n_fields * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    cck(cudaStreamSynchronize(st), "cv estimate");
  } catch (const CvFail& e) {
    return cfail(e.st, e.msg);
  }
  return RP_OK;
}

}  // extern "C"
