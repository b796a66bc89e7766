// CUDA kernels (sm_103a) of the stochastic spin-coherent-state trace:
// coherent-state sampling (Eqs. 15, 17-19), matrix-free H.psi fused with the
// Chebyshev recurrence (Eqs. 1-4, 13), the singlet Gram / exact time integral
// (Eqs. 20, 22) and the per-field averages with standard errors (Eqs. 18, 23).
#include "rp_kernels.cuh"

namespace rp {

namespace {

template <typename T>
struct Cx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ void cmac(Cx<T>& y, T ar, T ai, const Cx<T>& q) {
  // y += (ar + i ai) q
  y.re = fma(ar, q.re, fma(-ai, q.im, y.re));
  y.im = fma(ar, q.im, fma(ai, q.re, y.im));
}

template <typename T>
__device__ __forceinline__ void rmac(Cx<T>& y, T g, const Cx<T>& q) {
  y.re = fma(g, q.re, y.re);
  y.im = fma(g, q.im, y.im);
}

// Four complex values (the electron components of one nuclear configuration).
__device__ __forceinline__ void load4(const float* p, Cx<float> (&a)[4]) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + 1);
  a[0] = {u.x, u.y};
  a[1] = {u.z, u.w};
  a[2] = {v.x, v.y};
  a[3] = {v.z, v.w};
}
__device__ __forceinline__ void load4(const double* p, Cx<double> (&a)[4]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 u = __ldg(q + e);
    a[e] = {u.x, u.y};
  }
}
__device__ __forceinline__ void load4_rw(const float* p, Cx<float> (&a)[4]) {
  const float4 u = reinterpret_cast<const float4*>(p)[0];
  const float4 v = reinterpret_cast<const float4*>(p)[1];
  a[0] = {u.x, u.y};
  a[1] = {u.z, u.w};
  a[2] = {v.x, v.y};
  a[3] = {v.z, v.w};
}
__device__ __forceinline__ void load4_rw(const double* p, Cx<double> (&a)[4]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double2 u = q[e];
    a[e] = {u.x, u.y};
  }
}
__device__ __forceinline__ void store4(float* p, const Cx<float> (&a)[4]) {
  reinterpret_cast<float4*>(p)[0] = make_float4(a[0].re, a[0].im, a[1].re, a[1].im);
  reinterpret_cast<float4*>(p)[1] = make_float4(a[2].re, a[2].im, a[3].re, a[3].im);
}
__device__ __forceinline__ void store4(double* p, const Cx<double> (&a)[4]) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int e = 0; e < 4; ++e) q[e] = make_double2(a[e].re, a[e].im);
}

template <typename T>
__device__ __forceinline__ void store_singlet(T* x, const Cx<T> (&v)[4]) {
  // <S|v> = (v_{alpha beta} - v_{beta alpha}) / sqrt 2   (Eq. 3: P_S = |S><S|)
  const T r = T(0.70710678118654752440);
  x[0] = (v[1].re - v[2].re) * r;
  x[1] = (v[1].im - v[2].im) * r;
}

// y += Mx q on the electron of radical rr, Mx a 2x2 complex matrix (re/im arrays).
template <typename T>
__device__ __forceinline__ void apply_e2x2(Cx<T> (&y)[4], const Cx<T> (&q)[4], int rr,
                                           const T (&mr)[4], const T (&mi)[4]) {
  if (rr == 0) {
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
      cmac(y[e2], mr[0], mi[0], q[e2]);
      cmac(y[e2], mr[1], mi[1], q[2 + e2]);
      cmac(y[2 + e2], mr[2], mi[2], q[e2]);
      cmac(y[2 + e2], mr[3], mi[3], q[2 + e2]);
    }
  } else {
#pragma unroll
    for (int e1 = 0; e1 < 2; ++e1) {
      cmac(y[2 * e1], mr[0], mi[0], q[2 * e1]);
      cmac(y[2 * e1], mr[1], mi[1], q[2 * e1 + 1]);
      cmac(y[2 * e1 + 1], mr[2], mi[2], q[2 * e1]);
      cmac(y[2 * e1 + 1], mr[3], mi[3], q[2 * e1 + 1]);
    }
  }
}

// Partner contribution of nucleus p from configuration m + step * stride:
// step = +1 uses c U_p (I_+ brings M-1 to M), step = -1 uses c U_p^dagger.
template <typename T, bool ANISO>
__device__ __forceinline__ void add_partner(Cx<T> (&y)[4], const T* c, long long mp, int rr,
                                            const T* U, T coeff, bool up) {
  Cx<T> q[4];
  load4(c + mp * 8, q);
  if (!ANISO) {
    // isotropic: U = [[0, 0], [a/2, 0]], so only S_-I_+ / S_+I_- flip-flops
    const T g = coeff * U[4];
    if (rr == 0) {
      if (up) {
        rmac(y[2], g, q[0]);
        rmac(y[3], g, q[1]);
      } else {
        rmac(y[0], g, q[2]);
        rmac(y[1], g, q[3]);
      }
    } else {
      if (up) {
        rmac(y[1], g, q[0]);
        rmac(y[3], g, q[2]);
      } else {
        rmac(y[0], g, q[1]);
        rmac(y[2], g, q[3]);
      }
    }
  } else {
    T mr[4], mi[4];
    if (up) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        mr[i] = coeff * U[2 * i];
        mi[i] = coeff * U[2 * i + 1];
      }
    } else {  // U^dagger: (r, c) <- conj(U(c, r))
      const int tr[4] = {0, 2, 1, 3};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        mr[i] = coeff * U[2 * tr[i]];
        mi[i] = -coeff * U[2 * tr[i] + 1];
      }
    }
    apply_e2x2(y, q, rr, mr, mi);
  }
}

template <typename T>
__device__ __forceinline__ void add_field(T (&b1)[3], T (&b2)[3], int rr, T M, const T* v) {
  if (rr == 0) {
    b1[0] = fma(M, v[0], b1[0]);
    b1[1] = fma(M, v[1], b1[1]);
    b1[2] = fma(M, v[2], b1[2]);
  } else {
    b2[0] = fma(M, v[0], b2[0]);
    b2[1] = fma(M, v[1], b2[1]);
    b2[2] = fma(M, v[2], b2[2]);
  }
}

// One Chebyshev term for one nuclear configuration m of row blockIdx.y:
//   z = (H' - E_c) a / dE  with H' = H - i kappa (P_S - P_T),  a = phi_{n-1}(m, .)
//   FIRST: phi_1 = z,            acc = c_0 a + c_1 phi_1,  X[0] = <S|a>, X[1] = <S|phi_1>
//   MID:   phi_n = 2z - phi_{n-2}, acc += c_n phi_n,        X[n] = <S|phi_n>
//   LAST:  as MID but phi_n is not stored (acc becomes psi at the end of the step)
//   APPLY: next = s H' a - sh a   (used with s = 1, sh = i kbar/2 for H - iK)
template <typename T, bool ANISO>
__global__ void __launch_bounds__(256) k_cheb_step(
    const HamDev<T> H, const FieldDev<T>* __restrict__ fields, const int* __restrict__ row_field,
    const int* __restrict__ row_nmacro, long long macro, const T* __restrict__ cur,
    const T* __restrict__ prev, T* __restrict__ next, T* __restrict__ acc, T* __restrict__ X,
    const T* __restrict__ coef, int n_c, int n, int mode) {
  const long long Z = H.Z;
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (m >= Z) return;
  int f = 0;
  if (mode != MODE_APPLY) {
    if (macro >= row_nmacro[r]) return;
    f = row_field[r];
  }
  const FieldDev<T> F = fields[f];
  const size_t vs = (size_t)Z * 8;
  const T* c = cur + (size_t)r * vs;

  Cx<T> a[4];
  load4(c + m * 8, a);
  Cx<T> y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) y[e] = {T(0), T(0)};
  T b1[3] = {T(0), T(0), T(0)}, b2[3] = {T(0), T(0), T(0)};

  // spin-1/2 nuclei: digit j = bit p; exactly one partner
  for (int p = 0; p < H.n_half; ++p) {
    const int j = (int)((m >> p) & 1);
    const long long mp = j ? m - H.stride[p] : m + H.stride[p];
    const int rr = H.rad[p];
    add_field(b1, b2, rr, j ? T(-0.5) : T(0.5), H.v[p]);
    add_partner<T, ANISO>(y, c, mp, rr, H.U[p], T(1), j == 0);
  }
  // spin-1 nuclei: base-3 digits; partners +1 (j < 2) and -1 (j > 0), both sqrt 2
  long long qd = m >> H.n_half;
  for (int p = H.n_half; p < H.n_half + H.n_one; ++p) {
    const int j = (int)(qd % 3);
    qd /= 3;
    const int rr = H.rad[p];
    add_field(b1, b2, rr, T(1 - j), H.v[p]);
    const T s2 = T(1.41421356237309504880);
    if (j < 2) add_partner<T, ANISO>(y, c, m + H.stride[p], rr, H.U[p], s2, true);
    if (j > 0) add_partner<T, ANISO>(y, c, m - H.stride[p], rr, H.U[p], s2, false);
  }
  // any other spin
  for (int p = H.n_half + H.n_one; p < H.n_nuc; ++p) {
    const int d = H.d[p];
    const int j = (int)(qd % d);
    qd /= d;
    const int rr = H.rad[p];
    const T I = T(0.5) * T(d - 1), M = I - T(j);
    add_field(b1, b2, rr, M, H.v[p]);
    if (j < d - 1)
      add_partner<T, ANISO>(y, c, m + H.stride[p], rr, H.U[p], sqrt(I * (I + 1) - M * (M - 1)), true);
    if (j > 0)
      add_partner<T, ANISO>(y, c, m - H.stride[p], rr, H.U[p], sqrt(I * (I + 1) - M * (M + 1)), false);
  }

  // electron block: omega (S1z + S2z) + 2J S1.S2 - i kappa (2 P_S - 1)
  const T w = F.omega, Je = H.Je, kp = H.kappa, hJ = T(0.5) * Je;
  cmac(y[0], w + hJ, kp, a[0]);
  cmac(y[1], -hJ, T(0), a[1]);
  cmac(y[1], Je, kp, a[2]);
  cmac(y[2], Je, kp, a[1]);
  cmac(y[2], -hJ, T(0), a[2]);
  cmac(y[3], -w + hJ, kp, a[3]);
  // diagonal-in-m hyperfine part: (S1 . b1) x 1 + 1 x (S2 . b2), b_i = sum_k M_k A_k e_z
  {
    const T h = T(0.5);
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
      const Cx<T> lo = a[e2], hi = a[2 + e2];
      cmac(y[e2], h * b1[2], T(0), lo);
      cmac(y[e2], h * b1[0], -h * b1[1], hi);
      cmac(y[2 + e2], h * b1[0], h * b1[1], lo);
      cmac(y[2 + e2], -h * b1[2], T(0), hi);
    }
#pragma unroll
    for (int e1 = 0; e1 < 2; ++e1) {
      const Cx<T> lo = a[2 * e1], hi = a[2 * e1 + 1];
      cmac(y[2 * e1], h * b2[2], T(0), lo);
      cmac(y[2 * e1], h * b2[0], -h * b2[1], hi);
      cmac(y[2 * e1 + 1], h * b2[0], h * b2[1], lo);
      cmac(y[2 * e1 + 1], -h * b2[2], T(0), hi);
    }
  }
  // z = s y - sh a
  Cx<T> z[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    z[e].re = F.s * y[e].re - (F.sh_re * a[e].re - F.sh_im * a[e].im);
    z[e].im = F.s * y[e].im - (F.sh_re * a[e].im + F.sh_im * a[e].re);
  }
  const size_t off = (size_t)r * vs + (size_t)m * 8;
  if (mode == MODE_APPLY) {
    store4(next + off, z);
    return;
  }
  const T* cf = coef + (size_t)f * n_c * 2;
  T* xr = X + (size_t)r * n_c * Z * 2;
  if (mode == MODE_FIRST) {
    store4(next + off, z);
    const T c0r = cf[0], c0i = cf[1], c1r = cf[2], c1i = cf[3];
    Cx<T> s[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      s[e] = {T(0), T(0)};
      cmac(s[e], c0r, c0i, a[e]);
      cmac(s[e], c1r, c1i, z[e]);
    }
    store4(acc + off, s);
    store_singlet(xr + (size_t)m * 2, a);
    store_singlet(xr + ((size_t)Z + m) * 2, z);
    return;
  }
  Cx<T> pv[4];
  load4(prev + off, pv);
  Cx<T> ph[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ph[e].re = T(2) * z[e].re - pv[e].re;
    ph[e].im = T(2) * z[e].im - pv[e].im;
  }
  if (mode == MODE_MID) store4(next + off, ph);
  Cx<T> s[4];
  load4_rw(acc + off, s);
  const T cr = cf[2 * n], ci = cf[2 * n + 1];
#pragma unroll
  for (int e = 0; e < 4; ++e) cmac(s[e], cr, ci, ph[e]);
  store4(acc + off, s);
  store_singlet(xr + ((size_t)n * Z + m) * 2, ph);
}

// Singlet Gram G[r][n][m] += sum_z conj(x_n(z)) x_m(z) over a slice of z, for
// 4x4 tiles (n, m) with n <= m.  Products and per-chunk sums in T, running
// sums in FP64, one FP64 atomic per entry per CTA.
constexpr int kGramZC = 32;

template <typename T>
__global__ void k_gram(const T* __restrict__ X, double* __restrict__ G,
                       const int* __restrict__ row_nmacro, long long macro, long long Z, int n_c,
                       long long z_per_cta) {
  const int r = blockIdx.y;
  if (macro >= row_nmacro[r]) return;
  const long long z0 = (long long)blockIdx.x * z_per_cta;
  const long long z1 = min(Z, z0 + z_per_cta);
  if (z0 >= z1) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cx<T>* sx = reinterpret_cast<Cx<T>*>(smem_raw);  // [n_c][kGramZC]
  const int nt = n_c / 4;
  int ti = -1, tj = -1;
  {
    int k = threadIdx.x;
    for (int i = 0; i < nt; ++i) {
      const int cnt = nt - i;
      if (k < cnt) {
        ti = i;
        tj = i + k;
        break;
      }
      k -= cnt;
    }
  }
  double ar[4][4], ai[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.0;
  const T* Xr = X + (size_t)r * n_c * Z * 2;
  for (long long zc = z0; zc < z1; zc += kGramZC) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < n_c * kGramZC; idx += blockDim.x) {
      const int nn = idx / kGramZC, zz = idx % kGramZC;
      const long long z = zc + zz;
      Cx<T> v = {T(0), T(0)};
      if (z < z1) {
        v.re = Xr[((size_t)nn * Z + z) * 2];
        v.im = Xr[((size_t)nn * Z + z) * 2 + 1];
      }
      sx[nn * kGramZC + zz] = v;
    }
    __syncthreads();
    if (ti >= 0) {
      T pr[4][4], pi[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) pr[i][j] = pi[i][j] = T(0);
      for (int zz = 0; zz < kGramZC; ++zz) {
        Cx<T> xi[4], xj[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          xi[i] = sx[(4 * ti + i) * kGramZC + zz];
          xj[i] = sx[(4 * tj + i) * kGramZC + zz];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            pr[i][j] = fma(xi[i].re, xj[j].re, fma(xi[i].im, xj[j].im, pr[i][j]));
            pi[i][j] = fma(xi[i].re, xj[j].im, fma(-xi[i].im, xj[j].re, pi[i][j]));
          }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          ar[i][j] += (double)pr[i][j];
          ai[i][j] += (double)pi[i][j];
        }
    }
  }
  if (ti < 0) return;
  double* Gr = G + (size_t)r * n_c * n_c * 2;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int nn = 4 * ti + i, mm = 4 * tj + j;
      if (nn <= mm) {
        atomicAdd(Gr + ((size_t)nn * n_c + mm) * 2, ar[i][j]);
        atomicAdd(Gr + ((size_t)nn * n_c + mm) * 2 + 1, ai[i][j]);
      }
    }
}

template <int NT>
__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  return sh[0];
}

// integral[r] += sum_nm W_nm G_nm = sum_n W_nn G_nn + 2 Re sum_{n<m} W_nm G_nm; G := 0.
__global__ void __launch_bounds__(256) k_integrate(double* __restrict__ G,
                                                   const double* __restrict__ W,
                                                   const int* __restrict__ row_field,
                                                   const int* __restrict__ row_nmacro,
                                                   long long macro, int n_c,
                                                   double* __restrict__ integral) {
  __shared__ double sh[256];
  const int r = blockIdx.x;
  if (macro >= row_nmacro[r]) return;
  const int f = row_field[r];
  double* Gr = G + (size_t)r * n_c * n_c * 2;
  const double* Wf = W + (size_t)f * n_c * n_c * 2;
  double s = 0.0;
  for (int idx = threadIdx.x; idx < n_c * n_c; idx += blockDim.x) {
    const int nn = idx / n_c, mm = idx % n_c;
    if (nn > mm) continue;
    const double gr = Gr[2 * idx], gi = Gr[2 * idx + 1];
    const double v = Wf[2 * idx] * gr - Wf[2 * idx + 1] * gi;
    s += (nn == mm) ? v : 2.0 * v;
    Gr[2 * idx] = 0.0;
    Gr[2 * idx + 1] = 0.0;
  }
  const double tot = block_sum<256>(s, sh);
  if (threadIdx.x == 0) integral[r] += tot;
}

// survival[r] += |psi|^2 over a slice; psi of row r sits in S[n_macro % 2].
template <typename T>
__global__ void __launch_bounds__(256) k_norm(const T* __restrict__ S0, const T* __restrict__ S1,
                                              const int* __restrict__ row_nmacro, long long Z,
                                              long long z_per_cta, double* __restrict__ survival) {
  __shared__ double sh[256];
  const int r = blockIdx.y;
  const T* S = ((row_nmacro[r] & 1) ? S1 : S0) + (size_t)r * Z * 8;
  const long long z0 = (long long)blockIdx.x * z_per_cta;
  const long long z1 = min(Z, z0 + z_per_cta);
  double s = 0.0;
  for (long long m = z0 + threadIdx.x; m < z1; m += blockDim.x) {
    Cx<T> a[4];
    load4(S + m * 8, a);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      s += (double)a[e].re * (double)a[e].re + (double)a[e].im * (double)a[e].im;
  }
  const double tot = block_sum<256>(s, sh);
  if (threadIdx.x == 0) atomicAdd(survival + r, tot);
}

__global__ void k_finalize(RowsDev R, int rows, double k_S, double* __restrict__ per_sample) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const double phiS = k_S * R.integral[r];
  const double surv = R.survival[r];
  double* o = per_sample + (size_t)R.out[r] * 3;
  o[0] = phiS;
  o[1] = 1.0 - surv - phiS;  // Haberkorn: d|psi|^2/dt = -k_S <P_S> - k_T <P_T>
  o[2] = surv;
}

// Per field: mean of phi_S, phi_T (Eq. 18) and their standard errors
// sigma/sqrt(M) with the M-1 sample variance (Eq. 23), and mean survival.
__global__ void __launch_bounds__(256) k_stats(const double* __restrict__ per_sample, long long M,
                                               double* __restrict__ out) {
  __shared__ double sh[256];
  const int f = blockIdx.x;
  const double* p = per_sample + (size_t)f * M * 3;
  double s0 = 0, s1 = 0, s2 = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    s0 += p[3 * i];
    s1 += p[3 * i + 1];
    s2 += p[3 * i + 2];
  }
  const double m0 = block_sum<256>(s0, sh) / (double)M;
  __syncthreads();
  const double m1 = block_sum<256>(s1, sh) / (double)M;
  __syncthreads();
  const double m2 = block_sum<256>(s2, sh) / (double)M;
  __syncthreads();
  double v0 = 0, v1 = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    const double d0 = p[3 * i] - m0, d1 = p[3 * i + 1] - m1;
    v0 += d0 * d0;
    v1 += d1 * d1;
  }
  const double q0 = block_sum<256>(v0, sh);
  __syncthreads();
  const double q1 = block_sum<256>(v1, sh);
  if (threadIdx.x == 0) {
    const double den = (M > 1) ? (double)(M - 1) : 1.0;
    out[5 * f + 0] = m0;
    out[5 * f + 1] = m1;
    out[5 * f + 2] = sqrt(q0 / den / (double)M);
    out[5 * f + 3] = sqrt(q1 / den / (double)M);
    out[5 * f + 4] = m2;
  }
}

// ---- Philox4x32-10 (Salmon et al., SC'11) and coherent states (Eq. 15) ----

__device__ __forceinline__ void philox4x32_10(uint32_t (&c)[4], uint32_t k0, uint32_t k1) {
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

// One thread per (row, nucleus position): Philox draw of the direction
// (cos theta = 1 - 2 u1, phi = 2 pi u2; uniform on the sphere, Eq. 17) and the
// coherent-state components c_j = sqrt(C(2I, j)) cos^{2I-j}(theta/2)
// sin^j(theta/2) e^{i j phi}, j = I - M (Eq. 15 expanded in |I, M>).
__global__ void k_coherent_amps(const LayoutDev L, const long long* __restrict__ row_sample,
                                int rows, uint64_t seed, uint32_t pair, double* __restrict__ amps,
                                double* __restrict__ uv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * L.n_nuc) return;
  const int r = t / L.n_nuc, p = t % L.n_nuc;
  const int k = L.input_index[p];
  const unsigned long long s = (unsigned long long)row_sample[r];
  uint32_t c[4] = {(uint32_t)k, (uint32_t)(s & 0xFFFFFFFFull), (uint32_t)(s >> 32), pair};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
  if (uv) {
    uv[((size_t)r * L.n_nuc + k) * 2] = u1;
    uv[((size_t)r * L.n_nuc + k) * 2 + 1] = u2;
  }
  const double ch = sqrt(1.0 - u1), sh = sqrt(u1);  // cos(theta/2), sin(theta/2)
  const int d = L.d[p], twoI = d - 1;
  double* o = amps + ((size_t)r * kMaxNucDev + p) * 10 * 2;
  double binom = 1.0;  // C(2I, j)
  for (int j = 0; j < d; ++j) {
    if (j > 0) binom = binom * (double)(twoI - j + 1) / (double)j;
    double mag = sqrt(binom);
    for (int i = 0; i < twoI - j; ++i) mag *= ch;
    for (int i = 0; i < j; ++i) mag *= sh;
    double sn, cs;
    sincospi(2.0 * (double)j * u2, &sn, &cs);
    o[2 * j] = mag * cs;
    o[2 * j + 1] = mag * sn;
  }
}

// psi(m, e) = <e|S> prod_p c_p(j_p)  (Eq. 19), or the basis state |S, m0> (Eq. 13).
template <typename T>
__global__ void __launch_bounds__(256) k_init_state(const LayoutDev L,
                                                    const double* __restrict__ amps,
                                                    const long long* __restrict__ row_sample,
                                                    int deterministic, T* __restrict__ psi) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (m >= L.Z) return;
  double pr = 1.0, pi = 0.0;
  if (deterministic) {
    pr = (m == row_sample[r]) ? 1.0 : 0.0;
  } else {
    const double* A = amps + (size_t)r * kMaxNucDev * 10 * 2;
    long long q = m;
    for (int p = 0; p < L.n_nuc; ++p) {
      const int d = L.d[p];
      const int j = (int)(q % d);
      q /= d;
      const double ar = A[(p * 10 + j) * 2], ai = A[(p * 10 + j) * 2 + 1];
      const double nr = pr * ar - pi * ai;
      pi = pr * ai + pi * ar;
      pr = nr;
    }
  }
  const double s = 0.70710678118654752440;
  Cx<T> v[4];
  v[0] = {T(0), T(0)};
  v[1] = {(T)(s * pr), (T)(s * pi)};
  v[2] = {(T)(-s * pr), (T)(-s * pi)};
  v[3] = {T(0), T(0)};
  store4(psi + (size_t)r * L.Z * 8 + (size_t)m * 8, v);
}

__global__ void k_zero(double* p, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

inline unsigned grid1(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_coherent_amps(const LayoutDev& L, const long long* row_sample, int rows,
                                 uint64_t seed, uint32_t pair, double* amps, double* uv,
                                 cudaStream_t st) {
  const long long n = (long long)rows * L.n_nuc;
  if (n == 0) return cudaSuccess;
  k_coherent_amps<<<grid1(n, 128), 128, 0, st>>>(L, row_sample, rows, seed, pair, amps, uv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_state(const LayoutDev& L, const double* amps, const long long* row_sample,
                              int rows, int deterministic, T* psi, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int b = L.Z >= 256 ? 256 : (int)((L.Z + 31) / 32 * 32);
  dim3 grid(grid1(L.Z, b), rows);
  k_init_state<T><<<grid, b, 0, st>>>(L, amps, row_sample, deterministic, psi);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_step(const HamDev<T>& H, const FieldDev<T>* fields, const int* row_field,
                        const int* row_nmacro, long long macro, int rows, const T* cur,
                        const T* prev, T* next, T* acc, T* X, const T* coef, int n_c, int n,
                        int mode, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int b = H.Z >= 256 ? 256 : (int)((H.Z + 31) / 32 * 32);
  dim3 grid(grid1(H.Z, b), rows);
  if (H.aniso)
    k_cheb_step<T, true><<<grid, b, 0, st>>>(H, fields, row_field, row_nmacro, macro, cur, prev,
                                             next, acc, X, coef, n_c, n, mode);
  else
    k_cheb_step<T, false><<<grid, b, 0, st>>>(H, fields, row_field, row_nmacro, macro, cur, prev,
                                              next, acc, X, coef, n_c, n, mode);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram(const T* X, double* G, const int* row_nmacro, long long macro, int rows,
                        long long Z, int n_c, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int nt = n_c / 4;
  const int tiles = nt * (nt + 1) / 2;
  const int b = (tiles + 31) / 32 * 32;
  // aim for ~4 CTAs per SM over all rows, at least one chunk per CTA
  long long target = (4LL * 152 + rows - 1) / rows;
  long long chunks = (Z + kGramZC - 1) / kGramZC;
  long long split = target < 1 ? 1 : (target > chunks ? chunks : target);
  long long zper = (chunks + split - 1) / split * kGramZC;
  split = (Z + zper - 1) / zper;
  const size_t smem = (size_t)n_c * kGramZC * sizeof(Cx<T>);
  dim3 grid((unsigned)split, rows);
  k_gram<T><<<grid, b, smem, st>>>(X, G, row_nmacro, macro, Z, n_c, zper);
  return cudaGetLastError();
}

cudaError_t launch_integrate(double* G, const double* W, const int* row_field,
                             const int* row_nmacro, long long macro, int rows, int n_c,
                             double* integral, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_integrate<<<rows, 256, 0, st>>>(G, W, row_field, row_nmacro, macro, n_c, integral);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm(const T* S0, const T* S1, const int* row_nmacro, int rows, long long Z,
                        double* survival, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  long long zper = 256 * 16;
  dim3 grid(grid1(Z, (int)zper), rows);
  k_norm<T><<<grid, 256, 0, st>>>(S0, S1, row_nmacro, Z, zper, survival);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const RowsDev& R, int rows, double k_S, double* per_sample,
                            cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_finalize<<<grid1(rows, 128), 128, 0, st>>>(R, rows, k_S, per_sample);
  return cudaGetLastError();
}

cudaError_t launch_stats(const double* per_sample, int n_fields, long long M, double* out,
                         cudaStream_t st) {
  if (n_fields == 0) return cudaSuccess;
  k_stats<<<n_fields, 256, 0, st>>>(per_sample, M, out);
  return cudaGetLastError();
}

cudaError_t launch_zero(double* p, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_zero<<<grid1((long long)n, 256), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

template cudaError_t launch_init_state<float>(const LayoutDev&, const double*, const long long*,
                                              int, int, float*, cudaStream_t);
template cudaError_t launch_init_state<double>(const LayoutDev&, const double*, const long long*,
                                               int, int, double*, cudaStream_t);
template cudaError_t launch_step<float>(const HamDev<float>&, const FieldDev<float>*, const int*,
                                        const int*, long long, int, const float*, const float*,
                                        float*, float*, float*, const float*, int, int, int,
                                        cudaStream_t);
template cudaError_t launch_step<double>(const HamDev<double>&, const FieldDev<double>*,
                                         const int*, const int*, long long, int, const double*,
                                         const double*, double*, double*, double*, const double*,
                                         int, int, int, cudaStream_t);
template cudaError_t launch_gram<float>(const float*, double*, const int*, long long, int,
                                        long long, int, cudaStream_t);
template cudaError_t launch_gram<double>(const double*, double*, const int*, long long, int,
                                         long long, int, cudaStream_t);
template cudaError_t launch_norm<float>(const float*, const float*, const int*, int, long long,
                                        double*, cudaStream_t);
template cudaError_t launch_norm<double>(const double*, const double*, const int*, int, long long,
                                         double*, cudaStream_t);

}  // namespace rp
