// CUDA kernels (sm_103a) of the stochastic spin-coherent-state trace:
// coherent-state sampling (Eqs. 15, 17-19), matrix-free H.psi fused with the
// Chebyshev recurrence (Eqs. 1-4, 13), the singlet Gram / exact time integral
// (Eqs. 20, 22) and the per-field averages with standard errors (Eqs. 18, 23).
#include <algorithm>
#include <cstring>

#include "rp_kernels.cuh"
#include "rp_device.cuh"

namespace rp {

namespace {


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

// FP32: (re, im) as one packed pair (fma.rn.f32x2 of sm_100+, two fused
// multiply-adds per instruction).  Each lane rounds as fma() does, so results
// are bit-identical to the scalar form above.  (cmac stays scalar: its packed
// form needs the swapped pair (im, re) and measured slower.)
// The packed form of cmac for FP32 (same two rounding steps, bit-identical):
// y += (ar, -ai).(re, im) on the pair (q.im, q.re), then (ar, ar).(q.re, q.im).
// The pair (im, re) costs two moves; it pays where the coefficients are
// loop-invariant (the cluster kernel) and not elsewhere (measured).
__device__ __forceinline__ void cmac_packed(Cx<float>& y, float ar, float ai, const Cx<float>& q) {
  const float2 t = __ffma2_rn(make_float2(-ai, ai), make_float2(q.im, q.re),
                              make_float2(y.re, y.im));
  const float2 s = __ffma2_rn(make_float2(ar, ar), make_float2(q.re, q.im), t);
  y.re = s.x;
  y.im = s.y;
}

template <>
__device__ __forceinline__ void rmac<float>(Cx<float>& y, float g, const Cx<float>& q) {
  const float2 s = __ffma2_rn(make_float2(g, g), make_float2(q.re, q.im), make_float2(y.re, y.im));
  y.re = s.x;
  y.im = s.y;
}

// Four complex values (the electron components of one nuclear configuration):
// 32 bytes in FP32, moved with one 256-bit access per thread (sm_100+), so a
// warp reads or writes 1 KB contiguous per instruction; 64 bytes in FP64, two
// 256-bit accesses.  Addresses are 32-byte aligned (buffers are 256-byte
// aligned and a configuration is 32 or 64 bytes).
__device__ __forceinline__ void load4(const float* p, Cx<float> (&a)[4]) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a[0].re), "=f"(a[0].im), "=f"(a[1].re), "=f"(a[1].im), "=f"(a[2].re),
                 "=f"(a[2].im), "=f"(a[3].re), "=f"(a[3].im)
               : "l"(p));
}
__device__ __forceinline__ void load4(const double* p, Cx<double> (&a)[4]) {
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(a[0].re), "=d"(a[0].im), "=d"(a[1].re), "=d"(a[1].im)
               : "l"(p));
  asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(a[2].re), "=d"(a[2].im), "=d"(a[3].re), "=d"(a[3].im)
               : "l"(p + 4));
}
__device__ __forceinline__ void load4_rw(const float* p, Cx<float> (&a)[4]) {
  asm("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a[0].re), "=f"(a[0].im), "=f"(a[1].re), "=f"(a[1].im), "=f"(a[2].re),
                 "=f"(a[2].im), "=f"(a[3].re), "=f"(a[3].im)
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void load4_rw(const double* p, Cx<double> (&a)[4]) {
  asm("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(a[0].re), "=d"(a[0].im), "=d"(a[1].re), "=d"(a[1].im)
               : "l"(p)
               : "memory");
  asm("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];"
               : "=d"(a[2].re), "=d"(a[2].im), "=d"(a[3].re), "=d"(a[3].im)
               : "l"(p + 4)
               : "memory");
}
__device__ __forceinline__ void store4(float* p, const Cx<float> (&a)[4]) {
  asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a[0].re),
               "f"(a[0].im), "f"(a[1].re), "f"(a[1].im), "f"(a[2].re), "f"(a[2].im), "f"(a[3].re),
               "f"(a[3].im)
               : "memory");
}
__device__ __forceinline__ void store4(double* p, const Cx<double> (&a)[4]) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(a[0].re), "d"(a[0].im),
               "d"(a[1].re), "d"(a[1].im)
               : "memory");
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p + 4), "d"(a[2].re), "d"(a[2].im),
               "d"(a[3].re), "d"(a[3].im)
               : "memory");
}

// Shared-memory tile of a block's configurations in 16-byte planes: plane k
// holds bytes [16k, 16k + 16) of every configuration, so each 16-byte access
// of a warp is contiguous (no bank conflicts).
template <typename T>
struct Planes {
  static constexpr int kPlanes = (int)(4 * sizeof(Cx<T>) / 16);  // 2 (FP32) or 4 (FP64)
  static constexpr int kCx = 16 / (int)sizeof(Cx<T>);             // complex per plane entry
};

template <typename T>
__device__ __forceinline__ void tile_put(Cx<T>* tile, int nthreads, int i, const Cx<T> (&a)[4]) {
  constexpr int kc = Planes<T>::kCx;
#pragma unroll
  for (int k = 0; k < Planes<T>::kPlanes; ++k)
#pragma unroll
    for (int e = 0; e < kc; ++e) tile[((size_t)k * nthreads + i) * kc + e] = a[k * kc + e];
}

template <typename T>
__device__ __forceinline__ void tile_get(const Cx<T>* tile, int nthreads, int i, Cx<T> (&a)[4]) {
  constexpr int kc = Planes<T>::kCx;
#pragma unroll
  for (int k = 0; k < Planes<T>::kPlanes; ++k)
#pragma unroll
    for (int e = 0; e < kc; ++e) a[k * kc + e] = tile[((size_t)k * nthreads + i) * kc + e];
}

template <typename T>
__device__ __forceinline__ void store_singlet(T* x, const Cx<T> (&v)[4]) {
  // <S|v> = (v_{alpha beta} - v_{beta alpha}) / sqrt 2   (Eq. 3: P_S = |S><S|)
  const T r = T(0.70710678118654752440);
  x[0] = (v[1].re - v[2].re) * r;
  x[1] = (v[1].im - v[2].im) * r;
}

// Address of Re x_n(m) (Im is 4 floats further) of row r.
template <typename T>
__device__ __forceinline__ T* xblk_addr(T* X, int r, int n, unsigned m, long long Zs, int n_c) {
  const int row = 2 * n;
  return X + (size_t)r * xblk_row_floats(Zs, n_c) +
         (size_t)(m / kXChunk) * xrows_pad(n_c) * kXChunk + (row >> 3) * 128 +
         ((m % kXChunk) >> 2) * 32 + (row & 7) * 4 + (m & 3);
}

template <typename T>
__device__ __forceinline__ void store_singlet_blk(T* x, const Cx<T> (&v)[4]) {
  const T r = T(0.70710678118654752440);
  x[0] = (v[1].re - v[2].re) * r;
  x[4] = (v[1].im - v[2].im) * r;
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

// FP32 anisotropic spin-1/2 partner product on packed pairs: y += W q on the
// electron of radical rr, W = U_p (digit 0) or U_p^dagger (digit 1), with
// w[i] = (Re W_i, Re W_i, Im W_i, Im W_i) for entry i = 2 r + c.  The
// products with Re W accumulate in A and those with Im W in B, both on
// (re, im) pairs by fma.rn.f32x2 (two FMAs per instruction, no operand swap);
// y = A + i B is formed once per configuration by pack_combine.
template <int RR>
__device__ __forceinline__ void e2x2_packed_rr(float2 (&A)[4], float2 (&B)[4],
                                               const Cx<float> (&q)[4], const float4 (&w)[4]) {
  float2 qv[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) qv[e] = make_float2(q[e].re, q[e].im);
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    // RR = 0: outputs/inputs s and 2 + s; RR = 1: 2 s and 2 s + 1
    const int lo = RR == 0 ? s : 2 * s, hi = RR == 0 ? 2 + s : 2 * s + 1;
    A[lo] = __ffma2_rn(make_float2(w[0].x, w[0].y), qv[lo], A[lo]);
    B[lo] = __ffma2_rn(make_float2(w[0].z, w[0].w), qv[lo], B[lo]);
    A[lo] = __ffma2_rn(make_float2(w[1].x, w[1].y), qv[hi], A[lo]);
    B[lo] = __ffma2_rn(make_float2(w[1].z, w[1].w), qv[hi], B[lo]);
    A[hi] = __ffma2_rn(make_float2(w[2].x, w[2].y), qv[lo], A[hi]);
    B[hi] = __ffma2_rn(make_float2(w[2].z, w[2].w), qv[lo], B[hi]);
    A[hi] = __ffma2_rn(make_float2(w[3].x, w[3].y), qv[hi], A[hi]);
    B[hi] = __ffma2_rn(make_float2(w[3].z, w[3].w), qv[hi], B[hi]);
  }
}

// rr is the same for every thread (one nucleus): a uniform branch, and the
// register arrays keep compile-time indices.
__device__ __forceinline__ void e2x2_packed(float2 (&A)[4], float2 (&B)[4],
                                            const Cx<float> (&q)[4], int rr, const float4 (&w)[4]) {
  if (rr == 0) e2x2_packed_rr<0>(A, B, q, w);
  else e2x2_packed_rr<1>(A, B, q, w);
}

// y += A + i B (the packed partner sums of e2x2_packed).
__device__ __forceinline__ void pack_combine(Cx<float> (&y)[4], const float2 (&A)[4],
                                             const float2 (&B)[4]) {
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    y[e].re += A[e].x - B[e].y;
    y[e].im += A[e].y + B[e].x;
  }
}

// Fills the block's table of packed U_p / U_p^dagger entries of the spin-1/2
// nuclei p < n (8 n entries, the block's threads strided over them; barrier
// by the caller): wt[(2 p + j) 4 + i] = (Re, Re, Im, Im) of entry i of U_p
// (j = 0) or of U_p^dagger (j = 1; entry (r, c) = conj U_p(c, r)).
__device__ __forceinline__ void fill_wtab_entry(float4* wt, const HamDev<float>& H, int t) {
  const int p = t >> 3, jj = (t >> 2) & 1, i = t & 3;
  const int src = jj ? ((i & 1) << 1 | (i >> 1)) : i;
  const float re = H.U[p][2 * src], im = jj ? -H.U[p][2 * src + 1] : H.U[p][2 * src + 1];
  wt[(p * 2 + jj) * 4 + i] = make_float4(re, re, im, im);
}

__device__ __forceinline__ void fill_wtab_packed(float4* wt, const HamDev<float>& H, int n) {
  // at most two entries per thread: 8 n <= 2 blockDim for every block size
  // the launchers use (n <= log2 of the block for blocks below 256)
  const int t = (int)threadIdx.x;
  if (t < n * 8) fill_wtab_entry(wt, H, t);
  if (t + (int)blockDim.x < n * 8) fill_wtab_entry(wt, H, t + (int)blockDim.x);
}

// Partner contribution of nucleus p from configuration m + step * stride:
// step = +1 uses c U_p (I_+ brings M-1 to M), step = -1 uses c U_p^dagger.
template <typename T, bool ANISO>
__device__ __forceinline__ void add_partner_q(Cx<T> (&y)[4], const Cx<T> (&q)[4], int rr,
                                              const T* U, T coeff, bool up) {
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

template <typename T, bool ANISO>
__device__ __forceinline__ void add_partner(Cx<T> (&y)[4], const T* c, unsigned mp, int rr,
                                            const T* U, T coeff, bool up) {
  Cx<T> q[4];
  load4(c + (size_t)mp * 8, q);
  add_partner_q<T, ANISO>(y, q, rr, U, coeff, up);
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
// The block (a power of two, at most 256 configurations) stages its own
// configurations in shared memory: for the n_in innermost spin-1/2 nuclei
// (stride 2^p < blockDim) the partner m XOR 2^p lies in the same block.
// Configuration indices are 32-bit (Z <= 2^31); the nucleus loops are unrolled
// with predicates so per-nucleus constants are fixed-offset parameter loads.
constexpr int kStepThreads = 256;
constexpr int kInnerBits = 8;  // log2(kStepThreads)

// Isotropic flip-flop of a spin-1/2 nucleus: j = 0 (M = +1/2) takes the
// partner through U (y_beta += g q_alpha), j = 1 through U^dagger
// (y_alpha += g q_beta), g = a/2 on the electron of radical rr.
template <typename T>
__device__ __forceinline__ void iso_half(Cx<T> (&y)[4], const Cx<T> (&q)[4], int rr, unsigned j,
                                         T g) {
  const T gu = j ? T(0) : g, gd = j ? g : T(0);
  if (rr == 0) {
    rmac(y[0], gd, q[2]);
    rmac(y[1], gd, q[3]);
    rmac(y[2], gu, q[0]);
    rmac(y[3], gu, q[1]);
  } else {
    rmac(y[0], gd, q[1]);
    rmac(y[2], gd, q[3]);
    rmac(y[1], gu, q[0]);
    rmac(y[3], gu, q[2]);
  }
}

template <typename T, bool ANISO>
__device__ __forceinline__ void half_nucleus(Cx<T> (&y)[4], T (&b1)[3], T (&b2)[3],
                                             const HamDev<T>& H, int p, unsigned j,
                                             const Cx<T> (&q)[4]) {
  const int rr = H.rad[p];
  if (ANISO) {
    add_field(b1, b2, rr, j ? T(-0.5) : T(0.5), H.v[p]);
    add_partner_q<T, true>(y, q, rr, H.U[p], T(1), j == 0);
  } else {
    const T g = H.U[p][4];  // a/2
    const T dz = j ? -g : g;  // M a with M = +-1/2
    if (rr == 0) b1[2] += dz;
    else b2[2] += dz;
    iso_half(y, q, rr, j, g);
  }
}

// z = (H' a - E_c a) / dE from the partner sum y and the local fields b1, b2:
// adds the electron block omega (S1z + S2z) + 2J S1.S2 - i kappa (2 P_S - 1) and
// the diagonal-in-m hyperfine part (S1 . b1) x 1 + 1 x (S2 . b2),
// b_i = sum_k M_k A_k e_z, then applies the Chebyshev scaling of field F.
template <typename T, bool ANISO, bool PACKED = false>
__device__ __forceinline__ void finish_z(const HamDev<T>& H, const FieldDev<T>& F,
                                         const Cx<T> (&a)[4], Cx<T> (&y)[4], const T (&b1)[3],
                                         const T (&b2)[3], Cx<T> (&z)[4]) {
  // electron block: omega (S1z + S2z) + 2J S1.S2 - i kappa (2 P_S - 1), plus the
  // diagonal-in-m hyperfine part (S1 . b1) x 1 + 1 x (S2 . b2), b_i = sum_k M_k A_k e_z
  const T w = F.omega, Je = H.Je, kp = H.kappa, hJ = T(0.5) * Je;
  if (ANISO) {
    cmac(y[0], w + hJ, kp, a[0]);
    cmac(y[1], -hJ, T(0), a[1]);
    cmac(y[1], Je, kp, a[2]);
    cmac(y[2], Je, kp, a[1]);
    cmac(y[2], -hJ, T(0), a[2]);
    cmac(y[3], -w + hJ, kp, a[3]);
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
  } else if constexpr (PACKED) {
    const float sp = 0.5f * (b1[2] + b2[2]), sm = 0.5f * (b1[2] - b2[2]);
    cmac_packed(y[0], w + hJ + sp, kp, a[0]);
    cmac_packed(y[1], -hJ + sm, 0.f, a[1]);
    cmac_packed(y[1], Je, kp, a[2]);
    cmac_packed(y[2], Je, kp, a[1]);
    cmac_packed(y[2], -hJ - sm, 0.f, a[2]);
    cmac_packed(y[3], -w + hJ - sp, kp, a[3]);
  } else {
    const T sp = T(0.5) * (b1[2] + b2[2]), sm = T(0.5) * (b1[2] - b2[2]);
    cmac(y[0], w + hJ + sp, kp, a[0]);
    cmac(y[1], -hJ + sm, T(0), a[1]);
    cmac(y[1], Je, kp, a[2]);
    cmac(y[2], Je, kp, a[1]);
    cmac(y[2], -hJ - sm, T(0), a[2]);
    cmac(y[3], -w + hJ - sp, kp, a[3]);
  }
  // z = s y - sh a
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    z[e].re = F.s * y[e].re - (F.sh_re * a[e].re - F.sh_im * a[e].im);
    z[e].im = F.s * y[e].im - (F.sh_re * a[e].im + F.sh_im * a[e].re);
  }
}

// Chebyshev recurrence, accumulator and singlet slice of one configuration m
// of row r after the H' a partner sum y and local fields b1, b2 are known
// (see k_cheb_step for the modes).
template <typename T, bool ANISO>
__device__ __forceinline__ void term_epilogue(const HamDev<T>& H, const SysTab<T>& S,
                                              const FieldDev<T>& F, const Cx<T> (&a)[4],
                                              Cx<T> (&y)[4], const T (&b1)[3], const T (&b2)[3],
                                              int f, int r, unsigned m, size_t row0,
                                              const T* __restrict__ prev, T* __restrict__ next,
                                              T* __restrict__ acc, T* __restrict__ X,
                                              const T* __restrict__ coef, int n_c, int n,
                                              int mode, int xblk, const Cx<T>* pre_pv = nullptr,
                                              const Cx<T>* pre_acc = nullptr) {
  Cx<T> z[4];
  finish_z<T, ANISO>(H, F, a, y, b1, b2, z);
  const size_t off = row0 + (size_t)m * 8;
  if (mode == MODE_APPLY) {
    store4(next + off, z);
    return;
  }
  const T* cf = coef + (size_t)f * n_c * 4;  // c_n, then (FP32) c_n - fl(c_n)
  const T* cl = cf + 2 * n_c;
  const size_t Zs = (size_t)S.Zslot;
  T* xr = X + (size_t)r * n_c * Zs * 2;
  if (mode == MODE_FIRST) {
    store4(next + off, z);
    const T c0r = cf[0], c0i = cf[1], c1r = cf[2], c1i = cf[3];
    Cx<T> s[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      s[e] = {T(0), T(0)};
      if (sizeof(T) == 4) {
        cmac(s[e], cl[0], cl[1], a[e]);
        cmac(s[e], cl[2], cl[3], z[e]);
      }
      cmac(s[e], c0r, c0i, a[e]);
      cmac(s[e], c1r, c1i, z[e]);
    }
    store4(acc + off, s);
    if (xblk) {
      store_singlet_blk(xblk_addr(X, r, 0, m, S.Zslot, n_c), a);
      store_singlet_blk(xblk_addr(X, r, 1, m, S.Zslot, n_c), z);
    } else {
      store_singlet(xr + (size_t)m * 2, a);
      store_singlet(xr + (Zs + m) * 2, z);
    }
    return;
  }
  Cx<T> pv[4];
  if (pre_pv) {
#pragma unroll
    for (int e = 0; e < 4; ++e) pv[e] = pre_pv[e];
  } else {
    load4(prev + off, pv);
  }
  Cx<T> ph[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ph[e].re = T(2) * z[e].re - pv[e].re;
    ph[e].im = T(2) * z[e].im - pv[e].im;
  }
  if (mode == MODE_MID) store4(next + off, ph);
  Cx<T> s[4];
  if (pre_acc) {
#pragma unroll
    for (int e = 0; e < 4; ++e) s[e] = pre_acc[e];
  } else {
    load4_rw(acc + off, s);
  }
  const T cr = cf[2 * n], ci = cf[2 * n + 1];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (sizeof(T) == 4) cmac(s[e], cl[2 * n], cl[2 * n + 1], ph[e]);
    cmac(s[e], cr, ci, ph[e]);
  }
  store4(acc + off, s);
  if (xblk) store_singlet_blk(xblk_addr(X, r, n, m, S.Zslot, n_c), ph);
  else store_singlet(xr + ((size_t)n * Zs + m) * 2, ph);
}

// Body of one Chebyshev term; H is either the kernel-parameter copy (one
// system per launch) or a shared-memory copy of the row's system.  NH >= 0:
// a compiled shape (NH spin-1/2 then N1 spin-1 nuclei, nothing else, 256
// configurations per block), so every nucleus loop has fixed bounds and
// every per-nucleus constant a fixed offset.
template <typename T, bool ANISO, int NH = -1, int N1 = -1>
__device__ __forceinline__ void step_body(const HamDev<T>& H, const SysTab<T>& S, Cx<T>* tile,
                                          const FieldDev<T>* __restrict__ fields, int f, int r,
                                          const T* __restrict__ cur, const T* __restrict__ prev,
                                          T* __restrict__ next, T* __restrict__ acc,
                                          T* __restrict__ X, const T* __restrict__ coef, int n_c,
                                          int n, int mode, int xblk);

template <typename T, bool ANISO, bool MULTI, int NH = -1, int N1 = -1>
__global__ void __launch_bounds__(kStepThreads,
                                  sizeof(T) == 4 ? (ANISO ? 4 : (NH >= 0 ? 5 : 6)) : 2)
    k_cheb_step(
    const SysTab<T> S, const HamDev<T> H1, const FieldDev<T>* __restrict__ fields,
    const int* __restrict__ row_field, const int2* __restrict__ row_win, int macro_arg,
    const int* __restrict__ macro_dev, const T* __restrict__ cur, const T* __restrict__ prev,
    T* __restrict__ next, T* __restrict__ acc, T* __restrict__ X, const T* __restrict__ coef,
    int n_c, int n, int mode, int xblk) {
  extern __shared__ __align__(16) unsigned char step_smem[];
  Cx<T>* tile = reinterpret_cast<Cx<T>*>(step_smem);  // planes x blockDim x 16 B
  const int r = blockIdx.y;
  int f = 0;
  if (mode != MODE_APPLY) {
    const int macro = macro_dev ? *macro_dev : macro_arg;
    const int2 w = row_win[r];
    if (macro < w.x || macro >= w.y) return;  // the whole block: one row
    f = row_field[r];
  }
  if (MULTI) {
    __shared__ HamDev<T> Hs;  // constants of this row's system
    const int sidx = S.row_sys ? S.row_sys[r] : 0;
    const int4* src = reinterpret_cast<const int4*>(S.ham + sidx);
    int4* dst = reinterpret_cast<int4*>(&Hs);
    for (int i = threadIdx.x; i < (int)(sizeof(HamDev<T>) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    step_body<T, ANISO, NH, N1>(Hs, S, tile, fields, f, r, cur, prev, next, acc, X, coef, n_c, n,
                                mode, xblk);
  } else {
    step_body<T, ANISO, NH, N1>(H1, S, tile, fields, f, r, cur, prev, next, acc, X, coef, n_c, n,
                                mode, xblk);
  }
}

template <typename T, bool ANISO, int NH, int N1>
__device__ __forceinline__ void step_body(const HamDev<T>& H, const SysTab<T>& S, Cx<T>* tile,
                                          const FieldDev<T>* __restrict__ fields, int f, int r,
                                          const T* __restrict__ cur, const T* __restrict__ prev,
                                          T* __restrict__ next, T* __restrict__ acc,
                                          T* __restrict__ X, const T* __restrict__ coef, int n_c,
                                          int n, int mode, int xblk) {
  const unsigned Z = (unsigned)H.Z;
  const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = m < Z;
  const size_t row0 = (size_t)r * S.Zslot * 8;
  const T* c = cur + row0;
  const int nhalf = NH >= 0 ? NH : H.n_half;
  const int none = NH >= 0 ? N1 : H.n_one;
  const int nnuc = NH >= 0 ? NH + N1 : H.n_nuc;
  // spin-1/2 nuclei whose partner m XOR 2^p lies in this (power-of-two) block
  const int lb = 31 - __clz((int)blockDim.x);
  const int n_in = NH >= kInnerBits ? kInnerBits : (nhalf < lb ? nhalf : lb);

  Cx<T> a[4];
  if (valid) {
    load4(c + (size_t)m * 8, a);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) a[e] = {T(0), T(0)};
  }
  tile_put(tile, blockDim.x, threadIdx.x, a);
  // anisotropic FP64: W[p][j] = U_p (j = 0) and U_p^dagger (j = 1) of the
  // inner nuclei, entry (r, c) at 2 r + c, (re, im); FP32: the packed table
  // of every spin-1/2 nucleus (fill_wtab_packed)
  constexpr bool kPacked = ANISO && sizeof(T) == 4;
  __shared__ Cx<T> wtab[ANISO && !kPacked ? kInnerBits * 2 * 4 : 1];
  __shared__ float4 wtp[kPacked ? kMaxNucDev * 2 * 4 : 1];
  if (kPacked) {
    fill_wtab_packed(wtp, reinterpret_cast<const HamDev<float>&>(H), nhalf);
  } else if (ANISO) {
    // 8 n_in entries (40 with a 32-thread block and 5 inner nuclei): strided
    for (int t = (int)threadIdx.x; t < n_in * 8; t += (int)blockDim.x) {
      const int p = t >> 3, jj = (t >> 2) & 1, i = t & 3;
      const int src = jj ? ((i & 1) << 1 | (i >> 1)) : i;  // U^dagger(r, c) = conj U(c, r)
      const T re = H.U[p][2 * src], im = H.U[p][2 * src + 1];
      wtab[(p * 2 + jj) * 4 + i] = {re, jj ? -im : im};
    }
  }
  __syncthreads();
  if (!valid) {  // no barrier below
    // the tensor-core integral reads whole 16-configuration chunks: keep the
    // padding past Z at zero (a refilled row may hold a larger system's slices)
    if (xblk && mode != MODE_APPLY && m < ((Z + kXChunk - 1) / kXChunk) * kXChunk) {
      const Cx<T> zero[4] = {{T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}, {T(0), T(0)}};
      store_singlet_blk(xblk_addr(X, r, n, m, S.Zslot, n_c), zero);
      if (mode == MODE_FIRST) store_singlet_blk(xblk_addr(X, r, 0, m, S.Zslot, n_c), zero);
    }
    return;
  }

  Cx<T> y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) y[e] = {T(0), T(0)};
  T b1[3] = {T(0), T(0), T(0)}, b2[3] = {T(0), T(0), T(0)};

  if constexpr (kPacked) {
    // FP32 anisotropic: every spin-1/2 nucleus on packed pairs
    float2 A[4], B[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) A[e] = B[e] = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < kMaxNucDev; ++p) {
      if (p < nhalf) {
        const unsigned j = (m >> p) & 1u;
        Cx<float> q[4];
        if (p < kInnerBits) tile_get(tile, blockDim.x, threadIdx.x ^ (1u << p), q);
        else load4(c + (size_t)(m ^ (1u << p)) * 8, q);
        const float4* wp = wtp + (p * 2 + j) * 4;
        const float4 w[4] = {wp[0], wp[1], wp[2], wp[3]};
        add_field(b1, b2, H.rad[p], j ? T(-0.5) : T(0.5), H.v[p]);
        e2x2_packed(A, B, q, H.rad[p], w);
      }
    }
    pack_combine(reinterpret_cast<Cx<float>(&)[4]>(y), A, B);
  } else {
  // spin-1/2 nuclei inside the block: partner from shared memory
#pragma unroll
  for (int p = 0; p < kInnerBits; ++p) {
    if (p < n_in) {
      const unsigned j = (m >> p) & 1u;
      Cx<T> q[4];
      tile_get(tile, blockDim.x, threadIdx.x ^ (1u << p), q);
      if (ANISO) {
        // U_p (j = 0) or U_p^dagger (j = 1) from the block's table: two
        // vector loads instead of a select per matrix entry
        T mr[4], mi[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          mr[i] = wtab[(p * 2 + j) * 4 + i].re;
          mi[i] = wtab[(p * 2 + j) * 4 + i].im;
        }
        add_field(b1, b2, H.rad[p], j ? T(-0.5) : T(0.5), H.v[p]);
        apply_e2x2(y, q, H.rad[p], mr, mi);
      } else {
        half_nucleus<T, ANISO>(y, b1, b2, H, p, j, q);
      }
    }
  }
  // spin-1/2 nuclei outside the block (only when blockDim = 256): global
  // partner; the digit (m >> p) & 1 = (blockIdx.x >> (p - 8)) & 1 is the same
  // for the whole block, so the anisotropic form branches on it uniformly and
  // takes U_p or U_p^dagger straight from the constants
#pragma unroll
  for (int p = kInnerBits; p < kMaxNucDev; ++p) {
    if (p < nhalf) {
      const unsigned mp = m ^ (1u << p);
      Cx<T> q[4];
      load4(c + (size_t)mp * 8, q);
      if (ANISO) {
        if ((blockIdx.x >> (p - kInnerBits)) & 1u) {
          add_field(b1, b2, H.rad[p], T(-0.5), H.v[p]);
          add_partner_q<T, true>(y, q, H.rad[p], H.U[p], T(1), false);
        } else {
          add_field(b1, b2, H.rad[p], T(0.5), H.v[p]);
          add_partner_q<T, true>(y, q, H.rad[p], H.U[p], T(1), true);
        }
      } else {
        half_nucleus<T, ANISO>(y, b1, b2, H, p, (m >> p) & 1u, q);
      }
    }
  }
  }
  // spin-1 nuclei: base-3 digits; partners +1 (j < 2) and -1 (j > 0), both sqrt 2
  unsigned qd = m >> nhalf;
  const T s2 = T(1.41421356237309504880);
#pragma unroll 4
  for (int p = nhalf; p < nhalf + none; ++p) {
    const unsigned j = qd % 3u;
    qd /= 3u;
    const int rr = H.rad[p];
    const unsigned st = (unsigned)H.stride[p];
    if (ANISO) {
      add_field(b1, b2, rr, T(1) - T(j), H.v[p]);
    } else {
      const T dz = (T(1) - T(j)) * H.v[p][2];
      if (rr == 0) b1[2] += dz;
      else b2[2] += dz;
    }
    if (j < 2u) add_partner<T, ANISO>(y, c, m + st, rr, H.U[p], s2, true);
    if (j > 0u) add_partner<T, ANISO>(y, c, m - st, rr, H.U[p], s2, false);
  }
  // any other spin
  for (int p = nhalf + none; p < nnuc; ++p) {
    const unsigned d = (unsigned)H.d[p];
    const unsigned j = qd % d;
    qd /= d;
    const int rr = H.rad[p];
    const unsigned st = (unsigned)H.stride[p];
    const T I = T(0.5) * T(d - 1), M = I - T(j);
    add_field(b1, b2, rr, M, H.v[p]);
    if (j + 1u < d)
      add_partner<T, ANISO>(y, c, m + st, rr, H.U[p], sqrt(I * (I + 1) - M * (M - 1)), true);
    if (j > 0u)
      add_partner<T, ANISO>(y, c, m - st, rr, H.U[p], sqrt(I * (I + 1) - M * (M + 1)), false);
  }

  term_epilogue<T, ANISO>(H, S, fields[f], a, y, b1, b2, f, r, m, row0, prev, next, acc, X, coef,
                         n_c, n, mode, xblk);
}

// ---- FP32 term with the block's partner tiles staged by bulk async copies ----
//
// When every nucleus outside the innermost kInnerBits spin-1/2 positions has a
// stride that is a multiple of the block (n_half >= kInnerBits and 256
// configurations per block), the partner configurations m +- stride_p of a
// whole block form whole neighbouring blocks ("tiles") of the same row: one
// tile per outer spin-1/2 nucleus (m XOR 2^p), and one or two per outer nucleus
// of higher spin (digit j + 1 and j - 1 where they exist; the digit is the
// same for the whole tile).  One thread issues bulk copies (cp.async.bulk,
// completion counted on an mbarrier) of the block's own tile and of every
// partner tile at kernel start, so all of the block's reads of phi_{n-1} are in
// flight at once instead of one dependent 32-byte L2 load per partner and
// thread.  Tiles are kept as in memory (32 bytes per configuration); a thread
// reads entry t as two 16-byte halves in the order (t >> 2) & 1, which keeps
// each quarter-warp on distinct banks.
constexpr int kBulkTile = 256;                       // configurations per block
constexpr int kBulkTileBytes = kBulkTile * 32;       // FP32: 8 KB
constexpr int kBulkMaxSmem = 80 * 1024;              // own + partner tiles per block
constexpr long long kBulkWaitLimit = 1ll << 24;      // try_wait polls before giving up

__device__ __forceinline__ void tile_get_aos(const float* tile, unsigned t, Cx<float> (&q)[4]) {
  const unsigned sw = (t >> 2) & 1u;
  const float4* e = reinterpret_cast<const float4*>(tile) + 2 * t;
  const float4 u = e[sw], v = e[sw ^ 1u];
  const float4 lo = sw ? v : u, hi = sw ? u : v;
  q[0] = {lo.x, lo.y};
  q[1] = {lo.z, lo.w};
  q[2] = {hi.x, hi.y};
  q[3] = {hi.z, hi.w};
}

// Bounded wait for phase 0 of the block's mbarrier; false after the limit.
__device__ __forceinline__ bool bulk_wait(unsigned bar) {
  for (long long it = 0; it < kBulkWaitLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Partner tiles of tile c0 (first configuration), in the order the compute
// loop consumes them; calls emit(slot, first configuration of the partner).
// The digits of the outer nuclei are the same for every configuration of the
// tile, so they come from c0.
template <typename F>
__device__ __forceinline__ int bulk_partner_tiles(const HamDev<float>& H, unsigned c0, F&& emit) {
  int slot = 1;  // slot 0: the block's own tile
  for (int p = kInnerBits; p < H.n_half; ++p) emit(slot++, c0 ^ (1u << p));
  unsigned qd = c0 >> H.n_half;
  for (int p = H.n_half; p < H.n_nuc; ++p) {
    const unsigned d = (unsigned)H.d[p];
    const unsigned j = d == 3u ? qd % 3u : qd % d;
    qd = d == 3u ? qd / 3u : qd / d;
    const unsigned st = (unsigned)H.stride[p];
    if (j + 1u < d) emit(slot++, c0 + st);
    if (j > 0u) emit(slot++, c0 - st);
  }
  return slot;
}

template <bool ANISO>
__global__ void __launch_bounds__(kBulkTile, 2) k_cheb_step_bulk(
    const SysTab<float> S, const HamDev<float> H, const FieldDev<float>* __restrict__ fields,
    const int* __restrict__ row_field, const int2* __restrict__ row_win, int macro_arg,
    const int* __restrict__ macro_dev, const float* __restrict__ cur,
    const float* __restrict__ prev, float* __restrict__ next, float* __restrict__ acc,
    float* __restrict__ X, const float* __restrict__ coef, int n_c, int n, int mode, int xblk) {
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  __shared__ __align__(8) unsigned long long bar_storage[2];  // own tile, partner tiles
  const int r = blockIdx.y;
  int f = 0;
  if (mode != MODE_APPLY) {
    const int macro = macro_dev ? *macro_dev : macro_arg;
    const int2 w = row_win[r];
    if (macro < w.x || macro >= w.y) return;  // the whole block: one row
    f = row_field[r];
  }
  float* tiles = reinterpret_cast<float*>(bulk_smem);
  const unsigned bar_own = smem_u32(&bar_storage[0]), bar_part = smem_u32(&bar_storage[1]);
  const unsigned c0 = blockIdx.x * kBulkTile;
  const size_t row0 = (size_t)r * S.Zslot * 8;
  const float* c = cur + row0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_own) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_part) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    auto copy = [&](unsigned bar, int slot, unsigned first) {
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(tiles + (size_t)slot * kBulkTile * 8)),
          "l"(c + (size_t)first * 8), "r"((unsigned)kBulkTileBytes), "r"(bar)
          : "memory");
    };
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_own),
                 "r"((unsigned)kBulkTileBytes)
                 : "memory");
    copy(bar_own, 0, c0);
    const int n_tiles = bulk_partner_tiles(H, c0, [](int, unsigned) {});
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_part),
                 "r"((unsigned)((n_tiles - 1) * kBulkTileBytes))
                 : "memory");
    bulk_partner_tiles(H, c0, [&](int slot, unsigned first) { copy(bar_part, slot, first); });
  }
  const unsigned t = threadIdx.x;
  const unsigned m = c0 + t;
  const size_t off = row0 + (size_t)m * 8;
  // the streams this thread reads anyway, in flight during the tile copies
  Cx<float> pv[4], sa[4];
  const bool pre = mode == MODE_MID || mode == MODE_LAST;
  if (pre) {
    load4(prev + off, pv);
    load4_rw(acc + off, sa);
  }
  __shared__ float4 wtp[ANISO ? kMaxNucDev * 2 * 4 : 1];
  if (ANISO) fill_wtab_packed(wtp, H, H.n_half);
  __syncthreads();  // the barriers are initialised before anyone polls them
  if (!bulk_wait(bar_own) ) {
    if (S.err) atomicOr(S.err, 1);
    bulk_wait(bar_own);  // let copies still in flight land before the block exits
    bulk_wait(bar_part);
    return;
  }
  Cx<float> a[4];
  tile_get_aos(tiles, t, a);
  Cx<float> y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) y[e] = {0.f, 0.f};
  float b1[3] = {0.f, 0.f, 0.f}, b2[3] = {0.f, 0.f, 0.f};
  // anisotropic: the spin-1/2 products on packed pairs, in the same order as
  // k_cheb_step (results identical)
  float2 A[4], B[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) A[e] = B[e] = make_float2(0.f, 0.f);
  // spin-1/2 nuclei inside the tile
#pragma unroll
  for (int p = 0; p < kInnerBits; ++p) {
    Cx<float> q[4];
    tile_get_aos(tiles, t ^ (1u << p), q);
    const unsigned j = (m >> p) & 1u;
    if (ANISO) {
      const float4* wp = wtp + (p * 2 + j) * 4;
      const float4 w[4] = {wp[0], wp[1], wp[2], wp[3]};
      add_field(b1, b2, H.rad[p], j ? -0.5f : 0.5f, H.v[p]);
      e2x2_packed(A, B, q, H.rad[p], w);
    } else {
      half_nucleus<float, ANISO>(y, b1, b2, H, p, j, q);
    }
  }
  if (!bulk_wait(bar_part)) {
    if (S.err) atomicOr(S.err, 1);
    bulk_wait(bar_part);
    return;
  }
  // outer spin-1/2 nuclei: one partner tile each (slot 1 + p - kInnerBits)
#pragma unroll
  for (int p = kInnerBits; p < kMaxNucDev; ++p) {
    if (p < H.n_half) {
      Cx<float> q[4];
      tile_get_aos(tiles + (size_t)(1 + p - kInnerBits) * kBulkTile * 8, t, q);
      const unsigned j = (c0 >> p) & 1u;
      if (ANISO) {
        const float4* wp = wtp + (p * 2 + j) * 4;
        const float4 w[4] = {wp[0], wp[1], wp[2], wp[3]};
        add_field(b1, b2, H.rad[p], j ? -0.5f : 0.5f, H.v[p]);
        e2x2_packed(A, B, q, H.rad[p], w);
      } else {
        half_nucleus<float, ANISO>(y, b1, b2, H, p, j, q);
      }
    }
  }
  if (ANISO) pack_combine(y, A, B);
  // nuclei of higher spin: partners j + 1 (through U) and j - 1 (through U^dagger)
  int slot = 1 + H.n_half - kInnerBits;
  unsigned qd = c0 >> H.n_half;
  const float s2 = 1.41421356237309504880f;
#pragma unroll 4
  for (int p = H.n_half; p < H.n_half + H.n_one; ++p) {
    const unsigned j = qd % 3u;
    qd /= 3u;
    const int rr = H.rad[p];
    if (ANISO) {
      add_field(b1, b2, rr, 1.f - (float)j, H.v[p]);
    } else {
      const float dz = (1.f - (float)j) * H.v[p][2];
      if (rr == 0) b1[2] += dz;
      else b2[2] += dz;
    }
    if (j < 2u) {
      Cx<float> q[4];
      tile_get_aos(tiles + (size_t)(slot++) * kBulkTile * 8, t, q);
      add_partner_q<float, ANISO>(y, q, rr, H.U[p], s2, true);
    }
    if (j > 0u) {
      Cx<float> q[4];
      tile_get_aos(tiles + (size_t)(slot++) * kBulkTile * 8, t, q);
      add_partner_q<float, ANISO>(y, q, rr, H.U[p], s2, false);
    }
  }
  for (int p = H.n_half + H.n_one; p < H.n_nuc; ++p) {
    const unsigned d = (unsigned)H.d[p];
    const unsigned j = qd % d;
    qd /= d;
    const int rr = H.rad[p];
    const float I = 0.5f * (float)(d - 1), M = I - (float)j;
    add_field(b1, b2, rr, M, H.v[p]);
    if (j + 1u < d) {
      Cx<float> q[4];
      tile_get_aos(tiles + (size_t)(slot++) * kBulkTile * 8, t, q);
      add_partner_q<float, ANISO>(y, q, rr, H.U[p], sqrtf(I * (I + 1.f) - M * (M - 1.f)), true);
    }
    if (j > 0u) {
      Cx<float> q[4];
      tile_get_aos(tiles + (size_t)(slot++) * kBulkTile * 8, t, q);
      add_partner_q<float, ANISO>(y, q, rr, H.U[p], sqrtf(I * (I + 1.f) - M * (M + 1.f)), false);
    }
  }
  term_epilogue<float, ANISO>(H, S, fields[f], a, y, b1, b2, f, r, m, row0, prev, next, acc, X,
                              coef, n_c, n, mode, xblk, pre ? pv : nullptr,
                              pre ? sa : nullptr);
}

// Largest number of partner tiles over the tiles of a system (host side).
int bulk_max_partner_tiles(const HamDev<float>& H) {
  int t = H.n_half > kInnerBits ? H.n_half - kInnerBits : 0;
  for (int p = H.n_half; p < H.n_nuc; ++p) t += H.d[p] >= 3 ? 2 : 1;
  return t;
}

// ---- whole macro-steps of small systems in one CTA per row ----
// For Z <= kSmallMax (FP32 2048, FP64 1024 configurations) one CTA holds a
// row's phi_{n-1}, phi_{n-2} / phi_n and the accumulator in shared memory
// (16-byte planes) and runs every term of a macro-step between block
// barriers: each term reads the partners of every nucleus from shared memory,
// phi_{n-2} is read from the buffer that receives phi_n (same thread, same
// entry), and the singlet slices go to X for the Gram kernel as in k_cheb_step.
template <typename T>
struct SmallCfg {
  static constexpr int kMax = sizeof(T) == 4 ? 2048 : 1024;
  static constexpr int kThreads = 256;
};

template <typename T, bool ANISO>
__device__ __forceinline__ void apply_local(const HamDev<T>& H, const FieldDev<T>& F, unsigned m,
                                            const Cx<T> (&a)[4], const Cx<T>* buf, int nbuf,
                                            Cx<T> (&z)[4]) {
  Cx<T> y[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) y[e] = {T(0), T(0)};
  T b1[3] = {T(0), T(0), T(0)}, b2[3] = {T(0), T(0), T(0)};
  for (int p = 0; p < H.n_half; ++p) {
    const unsigned j = (m >> p) & 1u;
    Cx<T> q[4];
    tile_get(buf, nbuf, (int)(m ^ (1u << p)), q);
    half_nucleus<T, ANISO>(y, b1, b2, H, p, j, q);
  }
  unsigned qd = m >> H.n_half;
  const T s2 = T(1.41421356237309504880);
  for (int p = H.n_half; p < H.n_half + H.n_one; ++p) {
    const unsigned j = qd % 3u;
    qd /= 3u;
    const int rr = H.rad[p];
    const unsigned st = (unsigned)H.stride[p];
    if (ANISO) {
      add_field(b1, b2, rr, T(1) - T(j), H.v[p]);
    } else {
      const T dz = (T(1) - T(j)) * H.v[p][2];
      if (rr == 0) b1[2] += dz;
      else b2[2] += dz;
    }
    Cx<T> q[4];
    if (j < 2u) {
      tile_get(buf, nbuf, (int)(m + st), q);
      add_partner_q<T, ANISO>(y, q, rr, H.U[p], s2, true);
    }
    if (j > 0u) {
      tile_get(buf, nbuf, (int)(m - st), q);
      add_partner_q<T, ANISO>(y, q, rr, H.U[p], s2, false);
    }
  }
  for (int p = H.n_half + H.n_one; p < H.n_nuc; ++p) {
    const unsigned d = (unsigned)H.d[p];
    const unsigned j = qd % d;
    qd /= d;
    const int rr = H.rad[p];
    const unsigned st = (unsigned)H.stride[p];
    const T I = T(0.5) * T(d - 1), M = I - T(j);
    add_field(b1, b2, rr, M, H.v[p]);
    Cx<T> q[4];
    if (j + 1u < d) {
      tile_get(buf, nbuf, (int)(m + st), q);
      add_partner_q<T, ANISO>(y, q, rr, H.U[p], sqrt(I * (I + 1) - M * (M - 1)), true);
    }
    if (j > 0u) {
      tile_get(buf, nbuf, (int)(m - st), q);
      add_partner_q<T, ANISO>(y, q, rr, H.U[p], sqrt(I * (I + 1) - M * (M + 1)), false);
    }
  }
  finish_z<T, ANISO>(H, F, a, y, b1, b2, z);
}

template <typename T, bool ANISO>
__device__ __forceinline__ void macro_small_body(const HamDev<T>& H, const SysTab<T>& S,
                                                 const FieldDev<T>& F, int r,
                                                 const T* __restrict__ P, T* __restrict__ Q,
                                                 T* __restrict__ X, const T* __restrict__ cf,
                                                 int n_c) {
  extern __shared__ __align__(16) unsigned char small_smem[];
  const int Z = (int)H.Z;
  Cx<T>* bufA = reinterpret_cast<Cx<T>*>(small_smem);  // 4 complex per configuration
  Cx<T>* bufB = bufA + (size_t)4 * Z;
  Cx<T>* accb = bufB + (size_t)4 * Z;
  const size_t row0 = (size_t)r * S.Zslot * 8;
  const size_t Zs = (size_t)S.Zslot;
  T* xr = X + (size_t)r * n_c * Zs * 2;
  const T c0r = cf[0], c0i = cf[1];
  const T* cl = cf + 2 * n_c;  // (FP32) c_n - fl(c_n)
  for (int m = threadIdx.x; m < Z; m += blockDim.x) {
    Cx<T> a[4];
    load4(P + row0 + (size_t)m * 8, a);
    tile_put(bufA, Z, m, a);
    Cx<T> s[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      s[e] = {T(0), T(0)};
      if (sizeof(T) == 4) cmac(s[e], cl[0], cl[1], a[e]);
      cmac(s[e], c0r, c0i, a[e]);
    }
    tile_put(accb, Z, m, s);
    store_singlet(xr + (size_t)m * 2, a);
  }
  __syncthreads();
  for (int n = 1; n < n_c; ++n) {
    const Cx<T>* cur = (n & 1) ? bufA : bufB;  // phi_{n-1}
    Cx<T>* nxt = (n & 1) ? bufB : bufA;        // phi_{n-2}, then phi_n
    const T cr = cf[2 * n], ci = cf[2 * n + 1];
    for (int m = threadIdx.x; m < Z; m += blockDim.x) {
      Cx<T> a[4], z[4], ph[4];
      tile_get(cur, Z, m, a);
      apply_local<T, ANISO>(H, F, (unsigned)m, a, cur, Z, z);
      if (n == 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) ph[e] = z[e];
      } else {
        Cx<T> pv[4];
        tile_get(nxt, Z, m, pv);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ph[e].re = T(2) * z[e].re - pv[e].re;
          ph[e].im = T(2) * z[e].im - pv[e].im;
        }
      }
      Cx<T> s[4];
      tile_get(accb, Z, m, s);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (sizeof(T) == 4) cmac(s[e], cl[2 * n], cl[2 * n + 1], ph[e]);
        cmac(s[e], cr, ci, ph[e]);
      }
      tile_put(accb, Z, m, s);
      store_singlet(xr + ((size_t)n * Zs + m) * 2, ph);
      if (n < n_c - 1) tile_put(nxt, Z, m, ph);
    }
    __syncthreads();
  }
  for (int m = threadIdx.x; m < Z; m += blockDim.x) {
    Cx<T> s[4];
    tile_get(accb, Z, m, s);
    store4(Q + row0 + (size_t)m * 8, s);
  }
}

template <typename T, bool ANISO, bool MULTI>
__global__ void __launch_bounds__(256) k_macro_small(
    const SysTab<T> S, const HamDev<T> H1, const FieldDev<T>* __restrict__ fields,
    const int* __restrict__ row_field, const int2* __restrict__ row_win, int macro_arg,
    const int* __restrict__ macro_dev, const T* __restrict__ P, T* __restrict__ Q,
    T* __restrict__ X, const T* __restrict__ coef, int n_c) {
  const int r = blockIdx.x;
  const int macro = macro_dev ? *macro_dev : macro_arg;
  const int2 w = row_win[r];
  if (macro < w.x || macro >= w.y) return;
  const int f = row_field[r];
  const FieldDev<T> F = fields[f];
  const T* cf = coef + (size_t)f * n_c * 4;
  if (MULTI) {
    __shared__ HamDev<T> Hs;
    const int sidx = S.row_sys ? S.row_sys[r] : 0;
    const int4* src = reinterpret_cast<const int4*>(S.ham + sidx);
    int4* dst = reinterpret_cast<int4*>(&Hs);
    for (int i = threadIdx.x; i < (int)(sizeof(HamDev<T>) / 16); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    macro_small_body<T, ANISO>(Hs, S, F, r, P, Q, X, cf, n_c);
  } else {
    macro_small_body<T, ANISO>(H1, S, F, r, P, Q, X, cf, n_c);
  }
}

// ---- whole macro-steps of mid-size systems on a thread-block cluster ----
// For an isotropic FP32 system of spin-1/2 and spin-1 nuclei whose state
// splits over C = 2^c CTAs of one cluster (c <= kClusterMaxBits) with
// Zl = Z / C <= kClusterMaxLocal configurations per CTA, the cluster holds a
// row's phi_{n-1} and phi_n in distributed shared memory for a whole
// macro-step: HBM sees psi in, psi out and the singlet slices only.  The CTA
// rank is the value of the c outermost spin-1/2 nuclei (layout positions
// lb .. n_half - 1, lb = n_half - c), so the configuration of local index l is
//   m = ((l >> lb) << (lb + c)) | (rank << lb) | (l & (2^lb - 1)),
// and the partners of H.psi (Eq. 1, isotropic flip-flops) are
//   spin-1/2 at p < lb:  l XOR 2^p in this CTA,
//   spin-1/2 at lb + i:  the same l in CTA rank XOR 2^i (ld.shared::cluster),
//   spin-1 (p >= n_half): l +- stride_p / C in this CTA.
// Shared memory: two buffers of four planes (one per electron state e, Zl
// complex values each), so a flip-flop partner (two of the four components)
// costs two contiguous 8-byte reads per thread; then the accumulators
// psi(h) = sum_n c_n phi_n of every configuration but each thread's first,
// whose accumulator stays in registers.  Each thread owns the KPT local
// configurations l = tid + j NT; phi_{n-2} is read from the buffer that
// receives phi_n (same thread, same entry).  One cluster barrier per term
// orders the writes of phi_n before any CTA reads them and all reads of
// phi_{n-1} before the buffer is overwritten.  Control flow is uniform over
// the cluster: an inactive row returns in every CTA before the first barrier,
// and every thread of every CTA passes each barrier (the per-configuration
// work is predicated).
constexpr int kClusterMaxBits = 3;      // portable cluster sizes (<= 8 CTAs)
constexpr int kClusterMaxLocal = 2688;  // 64 Zl + 32 (Zl - NT) bytes of shared memory
constexpr int kClusterMaxIn = 12;       // inner spin-1/2 nuclei (2^12 > kClusterMaxLocal)
constexpr int kClusterMaxOne = 8;       // spin-1 nuclei (3^8 > kClusterMaxLocal)

// Per-system constants of the cluster kernel, by layout position (rad/us):
// radical bit masks, flip-flop couplings a/2 (spin-1/2) and sqrt(2) a/2
// (spin-1), the spin-1 diagonal a and the spin-1 local strides in bytes of a plane.
struct ClusterConst {
  int Zl, lb, cbits, n_one, NT;
  unsigned rr_in, rr_out, rr_one;
  float g_in[kClusterMaxIn];
  float g_out[kClusterMaxBits];
  float g_one[kClusterMaxOne];
  float v_one[kClusterMaxOne];
  unsigned st_one[kClusterMaxOne];
};

template <int KPT>
struct ClusterCfg {
  static constexpr int kNT = KPT == 1 ? 1024 : 896;
};

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Barrier over every thread of the cluster; release/acquire order the
// shared-memory writes of one term before the reads of the next.
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// The two halves of cluster_barrier, for work that needs neither (between them
// a thread may only touch memory no other CTA writes before the wait).
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}

// Complex values in shared memory (float2 = re, im).  Plain loads and stores,
// so the compiler keeps them ordered against the cluster barrier (its memory
// clobber) and schedules them freely between barriers; a peer CTA's shared
// memory is reached through a generic pointer from __cluster_map_shared_rank.
__device__ __forceinline__ Cx<float> ldc(const float2* p) {
  const float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ void stc(float2* p, const Cx<float>& v) { *p = make_float2(v.re, v.im); }
// Complex value at shared-memory byte address a of the CTA `rank` of this
// cluster (volatile: it stays between the cluster barriers around it).
__device__ __forceinline__ Cx<float> ld_peer(unsigned a, unsigned rank) {
  unsigned ra;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
  Cx<float> v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.re), "=f"(v.im) : "r"(ra));
  return v;
}

// Flip-flop of an isotropic nucleus on the electron of radical rr with the
// partner whose nuclear quantum number is one lower ("up": S_- I_+ brings it
// to this configuration) or one higher ("down"); g (u0, u1) goes to the two
// electron components it reaches.  Components read from the partner:
//   rr = 0: up (0, 1) -> y2, y3;  down (2, 3) -> y0, y1
//   rr = 1: up (0, 2) -> y1, y3;  down (1, 3) -> y0, y2
template <bool UP>
__device__ __forceinline__ void flip_add(Cx<float> (&y)[4], unsigned rr, float g,
                                         const Cx<float>& u0, const Cx<float>& u1) {
  if (rr == 0u) {
    rmac(y[UP ? 2 : 0], g, u0);
    rmac(y[UP ? 3 : 1], g, u1);
  } else {
    rmac(y[UP ? 1 : 0], g, u0);
    rmac(y[UP ? 3 : 2], g, u1);
  }
}

// Byte offsets (in units of one plane) of the two partner components read by
// a flip-flop (see flip_add).
template <bool UP>
__device__ __forceinline__ unsigned flip_p0(unsigned rr) { return UP ? 0u : (rr == 0u ? 2u : 1u); }
template <bool UP>
__device__ __forceinline__ unsigned flip_p1(unsigned rr) { return UP ? (rr == 0u ? 1u : 2u) : 3u; }

// Shape of a cluster instance: LB inner spin-1/2 nuclei, CB = log2 of the
// CTAs, N1 spin-1 nuclei, all known at compile time (LB >= 0), or read from
// ClusterConst (LB = -1: any shape the plan accepts).
template <int LB, int N1>
struct ClusterShape {
  static constexpr bool kStatic = LB >= 0;
  static constexpr int kIn = kStatic ? LB : kClusterMaxIn;     // unrolled inner nuclei
  static constexpr int kOne = kStatic ? N1 : kClusterMaxOne;   // unrolled spin-1 nuclei
  __host__ __device__ static constexpr int pow3(int n) { return n == 0 ? 1 : 3 * pow3(n - 1); }
  static constexpr unsigned kZl = kStatic ? (1u << (LB < 0 ? 0 : LB)) * pow3(N1 < 0 ? 0 : N1) : 0u;
};

// RR >= 0: the radical bit masks known at compile time, packed as
// rr_in | rr_out << 12 | rr_one << 15 (else read from ClusterConst).
template <int LB, int CB, int N1, int KPT, int RR = -1>
__global__ void __launch_bounds__(ClusterCfg<KPT>::kNT, 1) k_macro_cluster(
    const ClusterConst K, const HamDev<float> H, const FieldDev<float>* __restrict__ fields,
    const int* __restrict__ row_field, const int2* __restrict__ row_win, int macro_arg,
    const int* __restrict__ macro_dev, const float* __restrict__ P, float* __restrict__ Q,
    float* __restrict__ X, const float* __restrict__ coef, int n_c, long long Zslot, int xblk) {
  using Sh = ClusterShape<LB, N1>;
  extern __shared__ __align__(16) float2 cl_smem[];
  const int r = blockIdx.y;
  {
    const int macro = macro_dev ? *macro_dev : macro_arg;
    const int2 w = row_win[r];
    if (macro < w.x || macro >= w.y) return;  // the whole cluster: one row
  }
  const unsigned rank = cluster_rank();
  const unsigned Zl = Sh::kStatic ? Sh::kZl : (unsigned)K.Zl;
  const unsigned NT = (unsigned)K.NT;
  const int lb = Sh::kStatic ? LB : K.lb;
  const int cbits = Sh::kStatic ? CB : K.cbits;
  const int n_one = Sh::kStatic ? N1 : K.n_one;
  const unsigned lmask = (1u << lb) - 1u;
  // buffer b, plane e: cl_smem + (4 b + e) Zl; accumulators of l >= NT after
  // the two buffers, plane e at + e (Zl - NT)
  const unsigned apl = Zl > NT ? Zl - NT : 0u;
  float2* accs = cl_smem + 8u * Zl - NT;
  const unsigned sbase = smem_u32(cl_smem);
  const int f = row_field[r];
  const FieldDev<float> F = fields[f];
  const float* cf = coef + (size_t)f * n_c * 4;
  const float* cl = cf + 2 * n_c;  // c_n - fl(c_n)
  const float* Pr = P + (size_t)r * Zslot * 8;
  float* Qr = Q + (size_t)r * Zslot * 8;
  float* Xr = xblk ? X + (size_t)r * xblk_row_floats(Zslot, n_c) : X + (size_t)r * n_c * Zslot * 2;
  const unsigned tid = threadIdx.x;

  // configuration index and singlet-slice offset of each owned configuration
  unsigned mj[KPT], xj[KPT];
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const unsigned l = tid + j * NT;
    const unsigned m = ((l >> lb) << (lb + cbits)) | (rank << lb) | (l & lmask);
    mj[j] = m;
    xj[j] = xblk ? (m / kXChunk) * xrows_pad(n_c) * kXChunk + ((m % kXChunk) >> 2) * 32 + (m & 3)
                 : 2 * m;
  }
  // psi(t) of the row into buffer 0
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const unsigned l = tid + j * NT;
    if (l < Zl) {
      Cx<float> a[4];
      load4(Pr + (size_t)mj[j] * 8, a);
#pragma unroll
      for (int e = 0; e < 4; ++e) stc(cl_smem + e * Zl + l, a[e]);
    }
  }
  Cx<float> acc0[4];
  cluster_barrier();

  for (int n = 1; n < n_c; ++n) {
    const unsigned bo = ((n - 1) & 1) * 4u * Zl;  // phi_{n-1} in buffer (n - 1) % 2
    const float2* cur = cl_smem + bo;
    float2* oth = cl_smem + (4u * Zl - bo);        // phi_{n-2}, then phi_n
    const float cr = cf[2 * n], ci = cf[2 * n + 1], clr = cl[2 * n], cli = cl[2 * n + 1];
    // offset of slice n in a chunk (tensor-core layout) or of X[n] (plain)
    const unsigned xn = xblk ? ((2 * n) >> 3) * 128 + ((2 * n) & 7) * 4 : (unsigned)(2 * n * Zslot);
    const unsigned ximag = xblk ? 4u : 1u;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const unsigned l = tid + j * NT;
      if (l >= Zl) continue;
      Cx<float> a[4], y[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        a[e] = ldc(cur + e * Zl + l);
        y[e] = {0.f, 0.f};
      }
      float bz1 = 0.f, bz2 = 0.f;
      // spin-1/2 nuclei that select the CTA: partner in CTA rank XOR 2^i, the
      // direction is the same for the whole CTA
#pragma unroll
      for (int i = 0; i < (Sh::kStatic ? CB : kClusterMaxBits); ++i) {
        if (Sh::kStatic || i < cbits) {
          const unsigned pc = sbase + (bo + l) * 8u, peer = rank ^ (1u << i);
          const unsigned rr = ((RR >= 0 ? ((unsigned)RR >> 12) & 7u : K.rr_out) >> i) & 1u;
          const float g = K.g_out[i];
          if ((rank >> i) & 1u) {
            flip_add<false>(y, rr, g, ld_peer(pc + flip_p0<false>(rr) * Zl * 8u, peer),
                            ld_peer(pc + flip_p1<false>(rr) * Zl * 8u, peer));
            if (rr == 0u) bz1 -= g;
            else bz2 -= g;
          } else {
            flip_add<true>(y, rr, g, ld_peer(pc + flip_p0<true>(rr) * Zl * 8u, peer),
                           ld_peer(pc + flip_p1<true>(rr) * Zl * 8u, peer));
            if (rr == 0u) bz1 += g;
            else bz2 += g;
          }
        }
      }
      // spin-1/2 nuclei inside the CTA: both directions weighted by the digit
#pragma unroll
      for (int p = 0; p < Sh::kIn; ++p) {
        if (Sh::kStatic || p < lb) {
          const unsigned jb = (l >> p) & 1u;
          const float2* q8 = cur + (l ^ (1u << p));
          const unsigned rr = ((RR >= 0 ? (unsigned)RR & 0xFFFu : K.rr_in) >> p) & 1u;
          const float g = K.g_in[p];
          const float gu = jb ? 0.f : g, gd = jb ? g : 0.f;
          const float dz = jb ? -g : g;
          if (rr == 0u) {
            const float2* q = q8 + jb * 2u * Zl;
            const Cx<float> q0 = ldc(q);
            const Cx<float> q1 = ldc(q + Zl);
            rmac(y[2], gu, q0);
            rmac(y[3], gu, q1);
            rmac(y[0], gd, q0);
            rmac(y[1], gd, q1);
            bz1 += dz;
          } else {
            const float2* q = q8 + jb * Zl;
            const Cx<float> q0 = ldc(q);
            const Cx<float> q1 = ldc(q + 2u * Zl);
            rmac(y[1], gu, q0);
            rmac(y[3], gu, q1);
            rmac(y[0], gd, q0);
            rmac(y[2], gd, q1);
            bz2 += dz;
          }
        }
      }
      // spin-1 nuclei: base-3 digits of l >> lb (the digits of m >> n_half)
      unsigned qd = l >> lb;
#pragma unroll
      for (int i = 0; i < Sh::kOne; ++i) {
        if (Sh::kStatic || i < n_one) {
          const unsigned jd = qd % 3u;
          qd /= 3u;
          const unsigned rr = ((RR >= 0 ? ((unsigned)RR >> 15) & 0xFFu : K.rr_one) >> i) & 1u;
          const float g = K.g_one[i];
          const float dz = (1.f - (float)jd) * K.v_one[i];
          if (rr == 0u) bz1 += dz;
          else bz2 += dz;
          const unsigned st = Sh::kStatic ? (1u << LB) * ClusterShape<LB, N1>::pow3(i)
                                          : K.st_one[i] / 8u;
          if (jd < 2u) {
            const float2* q = cur + l + st;
            flip_add<true>(y, rr, g, ldc(q + flip_p0<true>(rr) * Zl), ldc(q + flip_p1<true>(rr) * Zl));
          }
          if (jd > 0u) {
            const float2* q = cur + l - st;
            flip_add<false>(y, rr, g, ldc(q + flip_p0<false>(rr) * Zl),
                            ldc(q + flip_p1<false>(rr) * Zl));
          }
        }
      }
      const float b1[3] = {0.f, 0.f, bz1}, b2[3] = {0.f, 0.f, bz2};
      Cx<float> z[4];
      finish_z<float, false, true>(H, F, a, y, b1, b2, z);
      Cx<float> ph[4], s[4];
      float2* al = accs + l;  // accumulator of l >= NT, plane e at + e apl
      if (n == 1) {
        const float c0r = cf[0], c0i = cf[1];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          ph[e] = z[e];
          s[e] = {0.f, 0.f};
          cmac_packed(s[e], cl[0], cl[1], a[e]);
          cmac_packed(s[e], c0r, c0i, a[e]);
        }
        float* x0 = Xr + xj[j];
        const float rs = 0.70710678118654752440f;
        x0[0] = (a[1].re - a[2].re) * rs;
        x0[ximag] = (a[1].im - a[2].im) * rs;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const Cx<float> pv = ldc(oth + e * Zl + l);
          ph[e].re = 2.f * z[e].re - pv.re;
          ph[e].im = 2.f * z[e].im - pv.im;
        }
        if (j == 0) {
#pragma unroll
          for (int e = 0; e < 4; ++e) s[e] = acc0[e];
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) s[e] = ldc(al + e * apl);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cmac_packed(s[e], clr, cli, ph[e]);
        cmac_packed(s[e], cr, ci, ph[e]);
      }
      if (j == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) acc0[e] = s[e];
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) stc(al + e * apl, s[e]);
      }
      if (n < n_c - 1) {
#pragma unroll
        for (int e = 0; e < 4; ++e) stc(oth + e * Zl + l, ph[e]);
      } else {
        float* xo = Xr + xj[j] + xn;
        const float rs = 0.70710678118654752440f;
        xo[0] = (ph[1].re - ph[2].re) * rs;
        xo[ximag] = (ph[1].im - ph[2].im) * rs;
      }
    }
    // The singlet slices of phi_n go to global memory between the arrive and
    // the wait, read back from this thread's own shared-memory entries (peers
    // only read them now): the release of the next term's arrive then finds
    // these stores long done instead of waiting for them.
    cluster_arrive();
    if (n < n_c - 1) {
      const float rs = 0.70710678118654752440f;
#pragma unroll
      for (int j = 0; j < KPT; ++j) {
        const unsigned l = tid + j * NT;
        if (l >= Zl) continue;
        const Cx<float> p1 = ldc(oth + 1u * Zl + l), p2 = ldc(oth + 2u * Zl + l);
        float* xo = Xr + xj[j] + xn;
        xo[0] = (p1.re - p2.re) * rs;
        xo[ximag] = (p1.im - p2.im) * rs;
      }
    }
    cluster_wait();
  }
  // psi(t + h) = the accumulator (no peer reads after the last barrier)
#pragma unroll
  for (int j = 0; j < KPT; ++j) {
    const unsigned l = tid + j * NT;
    if (l < Zl) {
      Cx<float> s[4];
      if (j == 0) {
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e] = acc0[e];
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) s[e] = ldc(accs + l + e * apl);
      }
      store4(Qr + (size_t)mj[j] * 8, s);
    }
  }
}

// Exact time integral of one macro-step (Eq. 20 / Eq. 22 over [t, t + h]):
//   integral[r] += sum_nm W_nm G_nm,  G_nm = sum_z conj(x_n(z)) x_m(z),
// where x_n = <S|phi_n> are the singlet slices stored by the step kernel.
// Each CTA forms the partial Gram of a slice of z for 4x4 tiles (n, m), n <= m
// (chunks of z staged z-major in shared memory; `groups` thread groups split
// each chunk), contracts it with W of the row's field in FP64 (factor 2 for
// n < m: W and G are Hermitian) and adds one scalar to integral[r].  Sums run
// in T within a chunk and in a second T accumulator across chunks.
constexpr int kGramThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kGramThreads) k_gram_integrate(
    const SysTab<T> S, const T* __restrict__ X, const double* __restrict__ W,
    const int* __restrict__ row_field, const int2* __restrict__ row_win, int macro_arg,
    const int* __restrict__ macro_dev, int n_c, int tiles, int groups, int zc,
    long long z_per_cta, double* __restrict__ integral) {
  const int r = blockIdx.y;
  const int macro = macro_dev ? *macro_dev : macro_arg;
  {
    const int2 w = row_win[r];
    if (macro < w.x || macro >= w.y) return;
  }
  const long long Z = S.ham[S.row_sys ? S.row_sys[r] : 0].Z;
  const long long Zs = S.Zslot;
  const long long z0 = (long long)blockIdx.x * z_per_cta;
  const long long z1 = min(Z, z0 + z_per_cta);
  if (z0 >= z1) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldn = n_c + 2;  // row stride of the z-major tile (16-byte multiple)
  Cx<T>* sx = reinterpret_cast<Cx<T>*>(smem_raw);  // [zc][ldn]
  const int tid = threadIdx.x;
  const int g = tid / tiles, t = tid % tiles;
  const bool active = g < groups;
  int ti = 0, tj = 0;
  {
    const int nt = n_c / 4;
    int k = t;
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
  T a2r[4][4], a2i[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) a2r[i][j] = a2i[i][j] = T(0);
  const T* Xr = X + (size_t)r * n_c * Zs * 2;
  for (long long c0 = z0; c0 < z1; c0 += zc) {
    __syncthreads();
    for (int idx = tid; idx < n_c * zc; idx += blockDim.x) {
      const int nn = idx / zc, zz = idx - nn * zc;
      const long long z = c0 + zz;
      Cx<T> v = {T(0), T(0)};
      if (z < z1) {
        v.re = Xr[((size_t)nn * Zs + z) * 2];
        v.im = Xr[((size_t)nn * Zs + z) * 2 + 1];
      }
      sx[zz * ldn + nn] = v;
    }
    __syncthreads();
    if (active) {
      T pr[4][4], pi[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) pr[i][j] = pi[i][j] = T(0);
      for (int zz = g; zz < zc; zz += groups) {
        const Cx<T>* row = sx + zz * ldn;
        Cx<T> xi[4], xj[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          xi[i] = row[4 * ti + i];
          xj[i] = row[4 * tj + i];
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
          a2r[i][j] += pr[i][j];
          a2i[i][j] += pi[i][j];
        }
    }
  }
  // combine the thread groups of each tile through shared memory
  __syncthreads();
  T* red = reinterpret_cast<T*>(smem_raw);  // [groups][tiles][32]
  if (active && groups > 1) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        red[((size_t)g * tiles + t) * 32 + 2 * (4 * i + j)] = a2r[i][j];
        red[((size_t)g * tiles + t) * 32 + 2 * (4 * i + j) + 1] = a2i[i][j];
      }
  }
  __syncthreads();
  double s = 0.0;
  if (active && g == 0) {
    const double* Wf = W + (size_t)row_field[r] * n_c * n_c * 2;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nn = 4 * ti + i, mm = 4 * tj + j;
        if (nn > mm) continue;
        double gr = (double)a2r[i][j], gi = (double)a2i[i][j];
        for (int q = 1; q < groups; ++q) {
          gr += (double)red[((size_t)q * tiles + t) * 32 + 2 * (4 * i + j)];
          gi += (double)red[((size_t)q * tiles + t) * 32 + 2 * (4 * i + j) + 1];
        }
        const size_t w = ((size_t)nn * n_c + mm) * 2;
        const double v = Wf[w] * gr - Wf[w + 1] * gi;
        s += (nn == mm) ? v : 2.0 * v;
      }
  }
  __syncthreads();
  double* sh = reinterpret_cast<double*>(smem_raw);
  const double tot = block_sum<kGramThreads>(s, sh);
  if (tid == 0) atomicAdd(integral + r, tot);
}

// Time-resolved observables (Eq. 18 for A = P_S, A = 1 and an electron
// operator A_e): after macro-step k, every row active in it holds psi(t_i),
// i = k + 1 - start, in Q; adds |<S|psi>|^2 (P_S = |S><S| on the electrons,
// identity on the nuclei), |psi|^2 and <psi| A_e x 1 |psi> over a slice of its
// configurations into trace[4 i .. 4 i + 3] (P_S, norm, Re, Im; FP64, summed
// over rows).
template <typename T>
__global__ void __launch_bounds__(256) k_trace(const SysTab<T> ST, const T* __restrict__ Q,
                                               const int2* __restrict__ row_win, int macro,
                                               long long z_per_cta, ElecOp A,
                                               double* __restrict__ trace) {
  __shared__ double sh[256];
  const int r = blockIdx.y;
  const int2 w = row_win[r];
  if (macro < w.x || macro >= w.y) return;
  const long long Z = ST.ham[ST.row_sys ? ST.row_sys[r] : 0].Z;
  const T* S = Q + (size_t)r * ST.Zslot * 8;
  const long long z0 = (long long)blockIdx.x * z_per_cta;
  const long long z1 = min(Z, z0 + z_per_cta);
  double ps = 0.0, nn = 0.0, ar = 0.0, ai = 0.0;
  for (long long m = z0 + threadIdx.x; m < z1; m += blockDim.x) {
    Cx<T> a[4];
    load4(S + m * 8, a);
    const double dr = (double)a[1].re - (double)a[2].re, di = (double)a[1].im - (double)a[2].im;
    ps += 0.5 * (dr * dr + di * di);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      nn += (double)a[e].re * (double)a[e].re + (double)a[e].im * (double)a[e].im;
    if (A.on) {
      // sum_e conj(a_e) (A a)_e
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        double yr = 0.0, yi = 0.0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const double xr = (double)a[f].re, xi = (double)a[f].im;
          yr += A.re[4 * e + f] * xr - A.im[4 * e + f] * xi;
          yi += A.re[4 * e + f] * xi + A.im[4 * e + f] * xr;
        }
        const double cr = (double)a[e].re, ci = (double)a[e].im;
        ar += cr * yr + ci * yi;
        ai += cr * yi - ci * yr;
      }
    }
  }
  const int i = macro + 1 - w.x;
  const double tps = block_sum<256>(ps, sh);
  if (threadIdx.x == 0) atomicAdd(trace + 4 * i, tps);
  __syncthreads();
  const double tnn = block_sum<256>(nn, sh);
  if (threadIdx.x == 0) atomicAdd(trace + 4 * i + 1, tnn);
  if (A.on) {
    __syncthreads();
    const double tar = block_sum<256>(ar, sh);
    if (threadIdx.x == 0) atomicAdd(trace + 4 * i + 2, tar);
    __syncthreads();
    const double tai = block_sum<256>(ai, sh);
    if (threadIdx.x == 0) atomicAdd(trace + 4 * i + 3, tai);
  }
}

// survival[r] += |psi|^2 over a slice for the flagged rows; psi of a row whose
// window ended at macro-step e sits in S[e % 2].
template <typename T>
__global__ void __launch_bounds__(256) k_norm(const SysTab<T> ST, const T* __restrict__ S0,
                                              const T* __restrict__ S1,
                                              const int2* __restrict__ row_win,
                                              const int* __restrict__ row_flag,
                                              long long z_per_cta, double* __restrict__ survival) {
  __shared__ double sh[256];
  const int r = blockIdx.y;
  if (row_flag && !row_flag[r]) return;
  const long long Z = ST.ham[ST.row_sys ? ST.row_sys[r] : 0].Z;
  const T* S = ((row_win[r].y & 1) ? S1 : S0) + (size_t)r * ST.Zslot * 8;
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

template <typename T>
__global__ void k_finalize(const SysTab<T> S, RowsDev R, int rows, double* __restrict__ per_sample) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows || (R.flag && !R.flag[r])) return;
  const double phiS = S.k_S[S.row_sys ? S.row_sys[r] : 0] * R.integral[r];
  const double surv = R.survival[r];
  double* o = per_sample + (size_t)R.out[r] * 3;
  o[0] = phiS;
  o[1] = 1.0 - surv - phiS;  // Haberkorn: d|psi|^2/dt = -k_S <P_S> - k_T <P_T>
  o[2] = surv;
}

// Per field: mean of phi_S, phi_T (Eq. 18) and their standard errors
// sigma/sqrt(M) with the M-1 sample variance (Eq. 23), and mean survival, over
// the samples per_sample[off[f] .. off[f] + cnt[f]).
__global__ void __launch_bounds__(256) k_stats(const double* __restrict__ per_sample,
                                               const long long* __restrict__ off,
                                               const long long* __restrict__ cnt,
                                               double* __restrict__ out) {
  __shared__ double sh[256];
  const int f = blockIdx.x;
  const double* p = per_sample + (size_t)off[f] * 3;
  const long long M = cnt[f];
  double s0 = 0, s1 = 0, s2 = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    s0 += p[3 * i];
    s1 += p[3 * i + 1];
    s2 += p[3 * i + 2];
  }
  const double Md = M > 0 ? (double)M : 1.0;
  const double m0 = block_sum<256>(s0, sh) / Md;
  __syncthreads();
  const double m1 = block_sum<256>(s1, sh) / Md;
  __syncthreads();
  const double m2 = block_sum<256>(s2, sh) / Md;
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
    out[5 * f + 2] = sqrt(q0 / den / Md);
    out[5 * f + 3] = sqrt(q1 / den / Md);
    out[5 * f + 4] = m2;
  }
}

// Deterministic trace from weighted propagations (Eq. 14 regrouped by J_z
// sector): out[f] = sum_i w_i (phi_S, phi_T, survival)_i, standard errors 0.
__global__ void __launch_bounds__(256) k_stats_weighted(const double* __restrict__ per_sample,
                                                        const long long* __restrict__ off,
                                                        const long long* __restrict__ cnt,
                                                        const double* __restrict__ w,
                                                        double* __restrict__ out) {
  __shared__ double sh[256];
  const int f = blockIdx.x;
  const double* p = per_sample + (size_t)off[f] * 3;
  const long long M = cnt[f];
  double s0 = 0, s1 = 0, s2 = 0;
  for (long long i = threadIdx.x; i < M; i += blockDim.x) {
    s0 += w[i] * p[3 * i];
    s1 += w[i] * p[3 * i + 1];
    s2 += w[i] * p[3 * i + 2];
  }
  const double m0 = block_sum<256>(s0, sh);
  __syncthreads();
  const double m1 = block_sum<256>(s1, sh);
  __syncthreads();
  const double m2 = block_sum<256>(s2, sh);
  if (threadIdx.x == 0) {
    out[5 * f + 0] = m0;
    out[5 * f + 1] = m1;
    out[5 * f + 2] = 0.0;
    out[5 * f + 3] = 0.0;
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

// Components c_j (o[2 j], o[2 j + 1], j = 0 .. 2I) of the coherent state of the
// nucleus at layout position p for sample s: Philox draw of the direction
// (counter (input index, s_lo, s_hi, pair), key seed; cos theta = 1 - 2 u1,
// phi = 2 pi u2, Eq. 17) and c_j = sqrt(C(2I, j)) cos^{2I-j}(theta/2)
// sin^j(theta/2) e^{i j phi} (Eq. 15); u receives (u1, u2).
__device__ __forceinline__ void coherent_amp(const LayoutDev& L, int p, uint32_t pair,
                                             unsigned long long s, uint64_t seed, double* o,
                                             double* u) {
  const int k = L.input_index[p];
  uint32_t c[4] = {(uint32_t)k, (uint32_t)(s & 0xFFFFFFFFull), (uint32_t)(s >> 32), pair};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
  u[0] = u1;
  u[1] = u2;
  const double ch = sqrt(1.0 - u1), sh = sqrt(u1);  // cos(theta/2), sin(theta/2)
  const int d = L.d[p], twoI = d - 1;
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

// One thread per (row, nucleus position): Philox draw of the direction
// (cos theta = 1 - 2 u1, phi = 2 pi u2; uniform on the sphere, Eq. 17) and the
// coherent-state components c_j = sqrt(C(2I, j)) cos^{2I-j}(theta/2)
// sin^j(theta/2) e^{i j phi}, j = I - M (Eq. 15 expanded in |I, M>).
template <typename T>
__global__ void k_coherent_amps(const SysTab<T> S, const long long* __restrict__ row_sample,
                                const int* __restrict__ row_flag, int rows, uint64_t seed,
                                double* __restrict__ amps, double* __restrict__ uv) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * kMaxNucDev) return;
  const int r = t / kMaxNucDev, p = t % kMaxNucDev;
  if (row_flag && !row_flag[r]) return;
  const int sidx = S.row_sys ? S.row_sys[r] : 0;
  const LayoutDev& L = S.lay[sidx];
  if (p >= L.n_nuc) return;
  const uint32_t pair = S.pair_of ? S.pair_of[sidx] : S.pair_base + (uint32_t)sidx;
  double* o = amps + ((size_t)r * kMaxNucDev + p) * 10 * 2;
  double u[2];
  coherent_amp(L, p, pair, (unsigned long long)row_sample[r], seed, o, u);
  if (uv) {
    const int k = L.input_index[p];
    uv[((size_t)r * L.n_nuc + k) * 2] = u[0];
    uv[((size_t)r * L.n_nuc + k) * 2 + 1] = u[1];
  }
}

// psi(m, e) = <e|S> prod_p c_p(j_p)  (Eq. 19), or the basis state |S, m0> (Eq. 13).
// Flagged rows only (all rows when row_flag is NULL); the state goes to
// S[start % 2] of the row's window, and the row's integral and survival restart.
template <typename T>
__global__ void __launch_bounds__(256) k_init_state(const SysTab<T> S,
                                                    const double* __restrict__ amps,
                                                    const long long* __restrict__ row_sample,
                                                    const int* __restrict__ row_flag,
                                                    const int2* __restrict__ row_win,
                                                    int deterministic, T* __restrict__ S0,
                                                    T* __restrict__ S1, double* __restrict__ integral,
                                                    double* __restrict__ survival) {
  const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (row_flag && !row_flag[r]) return;
  if (m == 0 && integral) {
    integral[r] = 0.0;
    survival[r] = 0.0;
  }
  const LayoutDev& L = S.lay[S.row_sys ? S.row_sys[r] : 0];
  if (m >= L.Z) return;
  T* psi = (row_win && (row_win[r].x & 1)) ? S1 : S0;
  double pr = 1.0, pi = 0.0;
  if (deterministic == 3) {
    // propagation i carries the i-th state |S, m> of every nuclear-M class
    const long long i = row_sample[r];
    pr = (S.sec_rank[m] == i) ? S.sec_scale[i] : 0.0;
  } else if (deterministic) {
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
  store4(psi + (size_t)r * S.Zslot * 8 + (size_t)m * 8, v);
}

// ---- one persistent launch over all work items of small systems ----
// Each CTA takes (system, field, sample) items from a device counter until
// none is left (device-side refill) and runs each item's whole propagation on
// chip: coherent-state amplitudes (Eqs. 15, 17, 19) and psi(0) in shared
// memory; per macro-step the n_c Chebyshev terms with the row in shared
// memory (as k_macro_small), the singlet slices in the CTA's own global
// scratch, and the exact time integral of the step (Eqs. 20, 22: partial
// Gram over 4 x 4 tiles (n, m), contracted with W in FP64); psi(h) becomes
// the next step's phi_0 by swapping buffers; at the end survival |psi(T)|^2,
// phi_S = k_S integral, phi_T = 1 - survival - phi_S into the per-sample
// output.  Items are independent, so no CTA waits for another.
constexpr int kPersistThreads = 256;
constexpr int kPersistGramZc = 32;  // configurations per staged Gram chunk

template <typename T>
size_t persist_smem_bytes(long long Zs, int n_c) {
  const int zc = sizeof(T) == 4 ? kPersistGramZc : kPersistGramZc / 2;
  return (size_t)3 * 4 * Zs * sizeof(Cx<T>) + (size_t)zc * (n_c + 2) * sizeof(Cx<T>);
}

template <typename T, bool ANISO>
__global__ void __launch_bounds__(kPersistThreads) k_persistent_small(
    const SysTab<T> S, const FieldDev<T>* __restrict__ fields, const T* __restrict__ coef,
    const double* __restrict__ W, const PItem* __restrict__ items, int n_items,
    int* __restrict__ counter, int n_c, int deterministic, uint64_t seed,
    T* __restrict__ Xscratch, double* __restrict__ per_sample) {
  extern __shared__ __align__(16) unsigned char psmem[];
  __shared__ HamDev<T> Hs;
  __shared__ double amps[kMaxNucDev * 10 * 2];
  __shared__ double red[kPersistThreads];
  __shared__ int s_item;
  const int Zs = (int)S.Zslot;
  const int zc = sizeof(T) == 4 ? kPersistGramZc : kPersistGramZc / 2;
  const int ldn = n_c + 2;
  Cx<T>* buf0 = reinterpret_cast<Cx<T>*>(psmem);
  Cx<T>* buf1 = buf0 + (size_t)4 * Zs;
  Cx<T>* buf2 = buf1 + (size_t)4 * Zs;
  Cx<T>* sx = buf2 + (size_t)4 * Zs;  // Gram staging [zc][ldn]
  T* xr = Xscratch + (size_t)blockIdx.x * n_c * Zs * 2;
  const int tid = threadIdx.x;
  // the 4 x 4 tile (ti, tj), ti <= tj, of the Gram this thread sums
  const int nt = n_c / 4, tiles = nt * (nt + 1) / 2;
  int ti = 0, tj = 0;
  {
    int q = tid % (tiles > 0 ? tiles : 1);
    for (int i = 0; i < nt; ++i) {
      const int cnt = nt - i;
      if (q < cnt) {
        ti = i;
        tj = i + q;
        break;
      }
      q -= cnt;
    }
  }
  const int groups = tiles >= kPersistThreads ? 1 : kPersistThreads / tiles;
  const int g = tid / (tiles > 0 ? tiles : 1);
  const bool tile_on = tid < tiles * groups;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;  // the same for the whole CTA
    const PItem I = items[it];
    {
      const int4* src = reinterpret_cast<const int4*>(S.ham + I.sys);
      int4* dst = reinterpret_cast<int4*>(&Hs);
      for (int i = tid; i < (int)(sizeof(HamDev<T>) / 16); i += blockDim.x) dst[i] = src[i];
    }
    const LayoutDev& L = S.lay[I.sys];
    if (!deterministic && tid < L.n_nuc) {
      double u[2];
      const uint32_t pair = S.pair_of ? S.pair_of[I.sys] : S.pair_base + (uint32_t)I.sys;
      coherent_amp(L, tid, pair, (unsigned long long)I.sample, seed, amps + tid * 20, u);
    }
    __syncthreads();
    const int Z = (int)Hs.Z;
    // psi(0) = |S> x prod_p c_p(j_p) (Eq. 19) or |S, m0> (Eq. 13) in buffer 0
    Cx<T>* P = buf0;   // phi_0 = psi(t)
    Cx<T>* B = buf1;   // phi_n of odd parity
    Cx<T>* A = buf2;   // accumulator psi(t + h)
    for (int m = tid; m < Z; m += blockDim.x) {
      double pr = 1.0, pi = 0.0;
      if (deterministic) {
        pr = (m == I.sample) ? 1.0 : 0.0;
      } else {
        int q = m;
        for (int p = 0; p < L.n_nuc; ++p) {
          const int d = L.d[p];
          const int j = q % d;
          q /= d;
          const double ar = amps[(p * 10 + j) * 2], ai = amps[(p * 10 + j) * 2 + 1];
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
      tile_put(P, Z, m, v);
    }
    __syncthreads();
    const FieldDev<T> F = fields[I.field];
    const T* cf = coef + (size_t)I.field * n_c * 4;
    const T* cl = cf + 2 * n_c;
    const double* Wf = W + (size_t)I.field * n_c * n_c * 2;
    double integral = 0.0;  // thread 0
    for (int km = 0; km < I.n_macro; ++km) {
      // ---- one macro-step: psi(t) in P, psi(t + h) into A, phi_n in P / B ----
      {
        const T c0r = cf[0], c0i = cf[1];
        for (int m = tid; m < Z; m += blockDim.x) {
          Cx<T> a[4];
          tile_get(P, Z, m, a);
          Cx<T> s4[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            s4[e] = {T(0), T(0)};
            if (sizeof(T) == 4) cmac(s4[e], cl[0], cl[1], a[e]);
            cmac(s4[e], c0r, c0i, a[e]);
          }
          tile_put(A, Z, m, s4);
          store_singlet(xr + (size_t)m * 2, a);
        }
        __syncthreads();
        for (int n = 1; n < n_c; ++n) {
          const Cx<T>* cur = (n & 1) ? P : B;  // phi_{n-1}
          Cx<T>* nxt = (n & 1) ? B : P;        // phi_{n-2}, then phi_n
          const T cr = cf[2 * n], ci = cf[2 * n + 1];
          for (int m = tid; m < Z; m += blockDim.x) {
            Cx<T> a[4], z[4], ph[4];
            tile_get(cur, Z, m, a);
            apply_local<T, ANISO>(Hs, F, (unsigned)m, a, cur, Z, z);
            if (n == 1) {
#pragma unroll
              for (int e = 0; e < 4; ++e) ph[e] = z[e];
            } else {
              Cx<T> pv[4];
              tile_get(nxt, Z, m, pv);
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                ph[e].re = T(2) * z[e].re - pv[e].re;
                ph[e].im = T(2) * z[e].im - pv[e].im;
              }
            }
            Cx<T> s4[4];
            tile_get(A, Z, m, s4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (sizeof(T) == 4) cmac(s4[e], cl[2 * n], cl[2 * n + 1], ph[e]);
              cmac(s4[e], cr, ci, ph[e]);
            }
            tile_put(A, Z, m, s4);
            store_singlet(xr + ((size_t)n * Zs + m) * 2, ph);
            if (n < n_c - 1) tile_put(nxt, Z, m, ph);
          }
          __syncthreads();
        }
      }
      // ---- exact time integral of the step: Re sum_nm W_nm G_nm ----
      {
        // sums in T within a chunk (pr_, pi_) and in a second T accumulator
        // across chunks (ar_, ai_), as in k_gram_integrate
        T ar_[4][4], ai_[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) ar_[i][j] = ai_[i][j] = T(0);
        for (int c0 = 0; c0 < Z; c0 += zc) {
          for (int idx = tid; idx < n_c * zc; idx += blockDim.x) {
            const int nn = idx / zc, zz = idx - nn * zc;
            const int z = c0 + zz;
            Cx<T> v = {T(0), T(0)};
            if (z < Z) {
              v.re = xr[((size_t)nn * Zs + z) * 2];
              v.im = xr[((size_t)nn * Zs + z) * 2 + 1];
            }
            sx[zz * ldn + nn] = v;
          }
          __syncthreads();
          if (tile_on) {
            T pr_[4][4], pi_[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) pr_[i][j] = pi_[i][j] = T(0);
            for (int zz = g; zz < zc; zz += groups) {
              const Cx<T>* row = sx + zz * ldn;
              Cx<T> xi[4], xj[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                xi[i] = row[4 * ti + i];
                xj[i] = row[4 * tj + i];
              }
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                  pr_[i][j] = fma(xi[i].re, xj[j].re, fma(xi[i].im, xj[j].im, pr_[i][j]));
                  pi_[i][j] = fma(xi[i].re, xj[j].im, fma(-xi[i].im, xj[j].re, pi_[i][j]));
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                ar_[i][j] += pr_[i][j];
                ai_[i][j] += pi_[i][j];
              }
          }
          __syncthreads();
        }
        double sum = 0.0;
        if (tile_on) {
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int nn = 4 * ti + i, mm = 4 * tj + j;
              if (nn > mm) continue;
              const size_t w = ((size_t)nn * n_c + mm) * 2;
              const double v = Wf[w] * (double)ar_[i][j] - Wf[w + 1] * (double)ai_[i][j];
              sum += (nn == mm) ? v : 2.0 * v;
            }
        }
        const double tot = block_sum<kPersistThreads>(sum, red);
        if (tid == 0) integral += tot;
        __syncthreads();
      }
      // psi(t + h) is phi_0 of the next step
      Cx<T>* t_ = P;
      P = A;
      A = t_;
    }
    double nn = 0.0;
    for (int m = tid; m < Z; m += blockDim.x) {
      Cx<T> a[4];
      tile_get(P, Z, m, a);
#pragma unroll
      for (int e = 0; e < 4; ++e)
        nn += (double)a[e].re * (double)a[e].re + (double)a[e].im * (double)a[e].im;
    }
    const double surv = block_sum<kPersistThreads>(nn, red);
    if (tid == 0) {
      const double phS = S.k_S[I.sys] * integral;
      per_sample[I.out * 3] = phS;
      per_sample[I.out * 3 + 1] = 1.0 - surv - phS;
      per_sample[I.out * 3 + 2] = surv;
    }
    __syncthreads();
  }
}

// Advances the device-side macro-step counter read by graph-replayed kernels.
__global__ void k_tick(int* macro_dev) { *macro_dev += 1; }

__global__ void k_zero(double* p, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = 0.0;
}

inline unsigned grid1(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

template <typename T>
cudaError_t launch_coherent_amps(const SysTab<T>& S, const long long* row_sample,
                                 const int* row_flag, int rows, uint64_t seed, double* amps,
                                 double* uv, cudaStream_t st) {
  const long long n = (long long)rows * kMaxNucDev;
  if (n == 0) return cudaSuccess;
  k_coherent_amps<T><<<grid1(n, 128), 128, 0, st>>>(S, row_sample, row_flag, rows, seed, amps, uv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_state(const SysTab<T>& S, const double* amps, const long long* row_sample,
                              const int* row_flag, const int2* row_win, int rows,
                              int deterministic, T* S0, T* S1, double* integral, double* survival,
                              cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int b = S.Zslot >= 256 ? 256 : (int)((S.Zslot + 31) / 32 * 32);
  dim3 grid(grid1(S.Zslot, b), rows);
  k_init_state<T><<<grid, b, 0, st>>>(S, amps, row_sample, row_flag, row_win, deterministic, S0,
                                      S1, integral, survival);
  return cudaGetLastError();
}

// The FP32 bulk kernel is only launched from launch_step<float>; the cast
// lets launch_step<double> compile the (never taken) branch.
template <typename T>
SysTab<float> S_as_float(const SysTab<T>& S) {
  return *reinterpret_cast<const SysTab<float>*>(&S);
}

template <typename T>
cudaError_t launch_step(const SysTab<T>& S, const HamDev<T>* one, int aniso, int bulk,
                        const FieldDev<T>* fields, const int* row_field, const int2* row_win,
                        int macro, const int* macro_dev, int rows, const T* cur, const T* prev,
                        T* next, T* acc, T* X, const T* coef, int n_c, int n, int mode,
                        int xblk, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  if (bulk && sizeof(T) == 4 && one && one->n_half >= kInnerBits && S.Zslot == one->Z &&
      one->Z % kBulkTile == 0) {
    const HamDev<float>& hf = *reinterpret_cast<const HamDev<float>*>(one);
    const size_t smem = (size_t)(1 + bulk_max_partner_tiles(hf)) * kBulkTileBytes;
    if (smem <= (size_t)kBulkMaxSmem) {
      static std::atomic<unsigned long long> attr_done[2];
      auto kf = aniso ? k_cheb_step_bulk<true> : k_cheb_step_bulk<false>;
      const cudaError_t e = smem_attr_once((const void*)kf, kBulkMaxSmem, attr_done[aniso ? 1 : 0]);
      if (e != cudaSuccess) return e;
      dim3 grid((unsigned)(one->Z / kBulkTile), rows);
      kf<<<grid, kBulkTile, smem, st>>>(
          S_as_float(S), hf, reinterpret_cast<const FieldDev<float>*>(fields), row_field, row_win,
          macro, macro_dev, reinterpret_cast<const float*>(cur),
          reinterpret_cast<const float*>(prev), reinterpret_cast<float*>(next),
          reinterpret_cast<float*>(acc), reinterpret_cast<float*>(X),
          reinterpret_cast<const float*>(coef), n_c, n, mode, xblk);
      return cudaGetLastError();
    }
  }
  // power-of-two blocks so that m XOR 2^p stays inside the block for 2^p < b
  int b = 32;
  while (b < kStepThreads && b < S.Zslot) b *= 2;
  const size_t smem = (size_t)b * 4 * sizeof(Cx<T>);
  dim3 grid(grid1(S.Zslot, b), rows);
  HamDev<T> h1;
  if (one) h1 = *one;
  else std::memset(&h1, 0, sizeof(h1));
  // compiled shape (fixed nucleus loops, 48 registers and 5 blocks per SM
  // instead of 40 and 6): 20 spin-1/2 nuclei, isotropic -- the paper's
  // Table I model, 3 % faster per term.  (The same for the 20-nucleus
  // anisotropic workload needs 67 registers, 3 blocks per SM, and measured
  // 12 % slower than the generic kernel at 4.)
  const bool t1_shape = one && !aniso && b == kStepThreads && one->n_half == 20 &&
                        one->n_nuc == 20;
  if (t1_shape) {
    k_cheb_step<T, false, false, 20, 0><<<grid, b, smem, st>>>(S, h1, fields, row_field, row_win,
                                                               macro, macro_dev, cur, prev, next,
                                                               acc, X, coef, n_c, n, mode, xblk);
  } else if (one) {
    if (aniso)
      k_cheb_step<T, true, false><<<grid, b, smem, st>>>(S, h1, fields, row_field, row_win, macro,
                                                         macro_dev, cur, prev, next, acc, X, coef,
                                                         n_c, n, mode, xblk);
    else
      k_cheb_step<T, false, false><<<grid, b, smem, st>>>(S, h1, fields, row_field, row_win, macro,
                                                          macro_dev, cur, prev, next, acc, X, coef,
                                                          n_c, n, mode, xblk);
  } else {
    if (aniso)
      k_cheb_step<T, true, true><<<grid, b, smem, st>>>(S, h1, fields, row_field, row_win, macro,
                                                        macro_dev, cur, prev, next, acc, X, coef,
                                                        n_c, n, mode, xblk);
    else
      k_cheb_step<T, false, true><<<grid, b, smem, st>>>(S, h1, fields, row_field, row_win, macro,
                                                         macro_dev, cur, prev, next, acc, X, coef,
                                                         n_c, n, mode, xblk);
  }
  return cudaGetLastError();
}

template <typename T>
int small_max_configs() {
  return SmallCfg<T>::kMax;
}

template <typename T>
cudaError_t launch_macro_small(const SysTab<T>& S, const HamDev<T>* one, int aniso,
                               const FieldDev<T>* fields, const int* row_field,
                               const int2* row_win, int macro, const int* macro_dev, int rows,
                               const T* P, T* Q, T* X, const T* coef, int n_c, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  if (S.Zslot > SmallCfg<T>::kMax) return cudaErrorInvalidValue;
  const size_t smem = (size_t)3 * 4 * S.Zslot * sizeof(Cx<T>);
  int b = 32;
  while (b < SmallCfg<T>::kThreads && b < S.Zslot) b *= 2;
  HamDev<T> h1;
  if (one) h1 = *one;
  else std::memset(&h1, 0, sizeof(h1));
#define RP_LAUNCH_SMALL(AN, MU)                                                                   \
  {                                                                                                \
    if (smem > 48 * 1024) {                                                                       \
      cudaError_t e = cudaFuncSetAttribute(k_macro_small<T, AN, MU>,                              \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
      if (e != cudaSuccess) return e;                                                            \
    }                                                                                              \
    k_macro_small<T, AN, MU><<<rows, b, smem, st>>>(S, h1, fields, row_field, row_win, macro,     \
                                                    macro_dev, P, Q, X, coef, n_c);                \
  }
  if (one) {
    if (aniso) RP_LAUNCH_SMALL(true, false) else RP_LAUNCH_SMALL(false, false)
  } else {
    if (aniso) RP_LAUNCH_SMALL(true, true) else RP_LAUNCH_SMALL(false, true)
  }
#undef RP_LAUNCH_SMALL
  return cudaGetLastError();
}

bool macro_cluster_plan(const HamDev<float>& H, ClusterPlan* out) {
  if (H.aniso || H.Z < 1 || H.n_half + H.n_one != H.n_nuc || H.n_one > kClusterMaxOne) return false;
  int c = -1;
  for (int b = 0; b <= kClusterMaxBits && b <= H.n_half; ++b)
    if ((H.Z >> b) <= kClusterMaxLocal) {
      c = b;
      break;
    }
  if (c < 0 || H.n_half - c > kClusterMaxIn) return false;
  ClusterPlan P;
  P.cbits = c;
  P.local = (int)(H.Z >> c);
  P.kpt = P.local <= 1024 ? 1 : (P.local <= 1792 ? 2 : 3);
  P.threads = ((P.local + P.kpt - 1) / P.kpt + 31) / 32 * 32;
  P.smem = (size_t)64 * P.local + (size_t)32 * (P.local > P.threads ? P.local - P.threads : 0);
  if (out) *out = P;
  return true;
}

namespace {

ClusterConst cluster_const(const HamDev<float>& H, const ClusterPlan& cp) {
  ClusterConst K;
  std::memset(&K, 0, sizeof(K));
  K.Zl = cp.local;
  K.cbits = cp.cbits;
  K.lb = H.n_half - cp.cbits;
  K.n_one = H.n_one;
  K.NT = cp.threads;
  for (int p = 0; p < H.n_nuc; ++p) {
    const unsigned rr = H.rad[p] ? 1u : 0u;
    if (p < K.lb) {
      K.rr_in |= rr << p;
      K.g_in[p] = H.U[p][4];
    } else if (p < H.n_half) {
      const int i = p - K.lb;
      K.rr_out |= rr << i;
      K.g_out[i] = H.U[p][4];
    } else {
      const int i = p - H.n_half;
      K.rr_one |= rr << i;
      K.g_one[i] = 1.41421356237309504880f * H.U[p][4];
      K.v_one[i] = H.v[p][2];
      K.st_one[i] = (unsigned)((H.stride[p] >> cp.cbits) * 8);
    }
  }
  return K;
}

template <int LB, int CB, int N1, int KPT, int RR = -1>
cudaError_t cluster_attr(std::atomic<unsigned long long>& done) {
  // the largest dynamic shared memory any launch of this instance asks for
  return smem_attr_once((const void*)k_macro_cluster<LB, CB, N1, KPT, RR>, 232448 - 1024, done);
}

std::atomic<unsigned long long> g_cluster_attr[5];

cudaLaunchConfig_t cluster_cfg(const ClusterPlan& cp, int rows, cudaStream_t st,
                               cudaLaunchAttribute* at) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(1u << cp.cbits, (unsigned)rows, 1);
  cfg.blockDim = dim3((unsigned)cp.threads, 1, 1);
  cfg.dynamicSmemBytes = cp.smem;
  cfg.stream = st;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1u << cp.cbits;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Instance of a plan: 3 for the compiled shape (5 inner spin-1/2 nuclei, 8
// CTAs, 4 spin-1 nuclei: the 12-nucleus workload with Z = 20736), else the
// generic instance of its configurations per thread (0, 1, 2).
constexpr int kRR534 = 0 | (7 << 12) | (12 << 15);  // radicals of the compiled 5/3/4 instance

int cluster_instance(const ClusterPlan& cp, const HamDev<float>& H) {
  if (H.n_half - cp.cbits == 5 && cp.cbits == 3 && H.n_one == 4 && cp.kpt == 3) {
    const ClusterConst K = cluster_const(H, cp);
    const int rr = (int)(K.rr_in | (K.rr_out << 12) | (K.rr_one << 15));
    return rr == kRR534 ? 4 : 3;
  }
  return cp.kpt - 1;
}

}  // namespace

cudaError_t launch_macro_cluster(const HamDev<float>& H, const FieldDev<float>* fields,
                                 const int* row_field, const int2* row_win, int macro,
                                 const int* macro_dev, int rows, const float* P, float* Q,
                                 float* X, const float* coef, int n_c, long long Zslot, int xblk,
                                 cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  ClusterPlan cp;
  if (!macro_cluster_plan(H, &cp)) return cudaErrorNotSupported;
  const ClusterConst K = cluster_const(H, cp);
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(cp, rows, st, at);
  cudaError_t e = cudaSuccess;
#define RP_CL(LB_, CB_, N1_, KPT_, I_)                                                            \
  e = cluster_attr<LB_, CB_, N1_, KPT_>(g_cluster_attr[I_]);                                      \
  if (e == cudaSuccess)                                                                            \
    e = cudaLaunchKernelEx(&cfg, k_macro_cluster<LB_, CB_, N1_, KPT_>, K, H, fields, row_field,   \
                           row_win, macro, macro_dev, P, Q, X, coef, n_c, Zslot, xblk);
#define RP_CL2(LB_, CB_, N1_, KPT_, RR_, I_)                                                      \
  e = cluster_attr<LB_, CB_, N1_, KPT_, RR_>(g_cluster_attr[I_]);                                 \
  if (e == cudaSuccess)                                                                            \
    e = cudaLaunchKernelEx(&cfg, k_macro_cluster<LB_, CB_, N1_, KPT_, RR_>, K, H, fields,         \
                           row_field, row_win, macro, macro_dev, P, Q, X, coef, n_c, Zslot, xblk);
  switch (cluster_instance(cp, H)) {
    case 0: RP_CL(-1, -1, -1, 1, 0) break;
    case 1: RP_CL(-1, -1, -1, 2, 1) break;
    case 2: RP_CL(-1, -1, -1, 3, 2) break;
    case 3: RP_CL(5, 3, 4, 3, 3) break;
    default: RP_CL2(5, 3, 4, 3, kRR534, 4) break;
  }
#undef RP_CL
#undef RP_CL2
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

bool macro_cluster_default(const HamDev<float>& H) {
  ClusterPlan cp;
  return macro_cluster_plan(H, &cp) && cluster_instance(cp, H) >= 3;
}

int macro_cluster_max_active(const HamDev<float>& H) {
  ClusterPlan cp;
  if (!macro_cluster_plan(H, &cp)) return 0;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(cp, 1, nullptr, at);
  int n = 0;
  cudaError_t e = cudaSuccess;
#define RP_CL(LB_, CB_, N1_, KPT_, I_)                                                            \
  e = cluster_attr<LB_, CB_, N1_, KPT_>(g_cluster_attr[I_]);                                      \
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, k_macro_cluster<LB_, CB_, N1_, KPT_>, &cfg);
#define RP_CL2(LB_, CB_, N1_, KPT_, RR_, I_)                                                      \
  e = cluster_attr<LB_, CB_, N1_, KPT_, RR_>(g_cluster_attr[I_]);                                 \
  if (e == cudaSuccess)                                                                            \
    e = cudaOccupancyMaxActiveClusters(&n, k_macro_cluster<LB_, CB_, N1_, KPT_, RR_>, &cfg);
  switch (cluster_instance(cp, H)) {
    case 0: RP_CL(-1, -1, -1, 1, 0) break;
    case 1: RP_CL(-1, -1, -1, 2, 1) break;
    case 2: RP_CL(-1, -1, -1, 3, 2) break;
    case 3: RP_CL(5, 3, 4, 3, 3) break;
    default: RP_CL2(5, 3, 4, 3, kRR534, 4) break;
  }
#undef RP_CL
#undef RP_CL2
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
size_t persistent_smem(long long Zs, int n_c) {
  return persist_smem_bytes<T>(Zs, n_c);
}

template <typename T>
int persistent_ctas(long long Zs, int n_c, int aniso) {
  const size_t smem = persist_smem_bytes<T>(Zs, n_c);
  int dev = 0, n_sm = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  static std::atomic<unsigned long long> attr_done[2];
  auto kf = aniso ? k_persistent_small<T, true> : k_persistent_small<T, false>;
  if (smem_attr_once((const void*)kf, (int)persist_smem_bytes<T>(SmallCfg<T>::kMax, 88),
                     attr_done[aniso ? 1 : 0]) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, kPersistThreads, smem) !=
      cudaSuccess)
    return 0;
  return n_sm * std::max(per_sm, 1);
}

template <typename T>
cudaError_t launch_persistent_small(const SysTab<T>& S, int aniso, const FieldDev<T>* fields,
                                    const T* coef, const double* W, const PItem* items,
                                    int n_items, int* counter, int n_c, int deterministic,
                                    uint64_t seed, T* Xscratch, int ctas, double* per_sample,
                                    cudaStream_t st) {
  if (n_items == 0 || ctas == 0) return cudaSuccess;
  if (S.Zslot > SmallCfg<T>::kMax) return cudaErrorInvalidValue;
  if (n_c % 4 != 0 || n_c > 88) return cudaErrorInvalidValue;  // <= 253 Gram tiles
  const size_t smem = persist_smem_bytes<T>(S.Zslot, n_c);
  auto kf = aniso ? k_persistent_small<T, true> : k_persistent_small<T, false>;
  // the shared-memory attribute was set by persistent_ctas, which gave `ctas`
  kf<<<ctas, kPersistThreads, smem, st>>>(S, fields, coef, W, items, n_items, counter, n_c,
                                          deterministic, seed, Xscratch, per_sample);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram_integrate(const SysTab<T>& S, const T* X, const double* W,
                                  const int* row_field, const int2* row_win, int macro,
                                  const int* macro_dev, int rows, int n_c, double* integral,
                                  cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const int nt = n_c / 4;
  const int tiles = nt * (nt + 1) / 2;
  const int groups = tiles >= kGramThreads ? 1 : kGramThreads / tiles;
  const int zc = sizeof(T) == 4 ? 32 : 16;
  const long long z_per_cta = 1024;
  const size_t tile_b = (size_t)zc * (n_c + 2) * sizeof(Cx<T>);
  const size_t red_b = (size_t)groups * tiles * 32 * sizeof(T);
  size_t smem = tile_b > red_b ? tile_b : red_b;
  if (smem < kGramThreads * sizeof(double)) smem = kGramThreads * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_integrate<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)((S.Zslot + z_per_cta - 1) / z_per_cta), rows);
  k_gram_integrate<T><<<grid, kGramThreads, smem, st>>>(S, X, W, row_field, row_win, macro,
                                                        macro_dev, n_c, tiles, groups, zc,
                                                        z_per_cta, integral);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm(const SysTab<T>& S, const T* S0, const T* S1, const int2* row_win,
                        const int* row_flag, int rows, double* survival, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  long long zper = 256 * 16;
  dim3 grid(grid1(S.Zslot, (int)zper), rows);
  k_norm<T><<<grid, 256, 0, st>>>(S, S0, S1, row_win, row_flag, zper, survival);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finalize(const SysTab<T>& S, const RowsDev& R, int rows, double* per_sample,
                            cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  k_finalize<T><<<grid1(rows, 128), 128, 0, st>>>(S, R, rows, per_sample);
  return cudaGetLastError();
}

cudaError_t launch_stats(const double* per_sample, const long long* off, const long long* cnt,
                         int n_fields, double* out, cudaStream_t st) {
  if (n_fields == 0) return cudaSuccess;
  k_stats<<<n_fields, 256, 0, st>>>(per_sample, off, cnt, out);
  return cudaGetLastError();
}

cudaError_t launch_stats_weighted(const double* per_sample, const long long* off,
                                  const long long* cnt, const double* w, int n_fields,
                                  double* out, cudaStream_t st) {
  if (n_fields == 0) return cudaSuccess;
  k_stats_weighted<<<n_fields, 256, 0, st>>>(per_sample, off, cnt, w, out);
  return cudaGetLastError();
}

size_t xblk_floats_per_row(long long Zs, int n_c) { return xblk_row_floats(Zs, n_c); }

template <typename T>
cudaError_t launch_trace(const SysTab<T>& S, const T* Q, const int2* row_win, int macro, int rows,
                         const ElecOp& A, double* trace, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  const long long zper = 8192;
  dim3 grid(grid1(S.Zslot, (int)zper), rows);
  k_trace<T><<<grid, 256, 0, st>>>(S, Q, row_win, macro, zper, A, trace);
  return cudaGetLastError();
}

cudaError_t launch_tick(int* macro_dev, cudaStream_t st) {
  k_tick<<<1, 1, 0, st>>>(macro_dev);
  return cudaGetLastError();
}

cudaError_t launch_zero(double* p, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_zero<<<grid1((long long)n, 256), 256, 0, st>>>(p, n);
  return cudaGetLastError();
}

template cudaError_t launch_coherent_amps<float>(const SysTab<float>&, const long long*, const int*,
                                                 int, uint64_t, double*, double*, cudaStream_t);
template cudaError_t launch_init_state<float>(const SysTab<float>&, const double*, const long long*,
                                              const int*, const int2*, int, int, float*, float*, double*,
                                              double*, cudaStream_t);
template cudaError_t launch_step<float>(const SysTab<float>&, const HamDev<float>*, int, int,
                                        const FieldDev<float>*, const int*, const int2*, int,
                                        const int*, int, const float*, const float*, float*, float*, float*,
                                        const float*, int, int, int, int, cudaStream_t);
template cudaError_t launch_gram_integrate<float>(const SysTab<float>&, const float*, const double*,
                                                  const int*, const int2*, int, const int*, int,
                                                  int, double*, cudaStream_t);
template int small_max_configs<float>();
template size_t persistent_smem<float>(long long, int);
template int persistent_ctas<float>(long long, int, int);
template cudaError_t launch_persistent_small<float>(const SysTab<float>&, int, const FieldDev<float>*,
                                                    const float*, const double*, const PItem*, int,
                                                    int*, int, int, uint64_t, float*, int, double*,
                                                    cudaStream_t);
template cudaError_t launch_macro_small<float>(const SysTab<float>&, const HamDev<float>*, int,
                                               const FieldDev<float>*, const int*, const int2*, int,
                                               const int*, int, const float*, float*, float*,
                                               const float*, int, cudaStream_t);
template cudaError_t launch_norm<float>(const SysTab<float>&, const float*, const float*, const int2*,
                                        const int*, int, double*, cudaStream_t);
template cudaError_t launch_trace<float>(const SysTab<float>&, const float*, const int2*, int, int,
                                         const ElecOp&, double*, cudaStream_t);
template cudaError_t launch_finalize<float>(const SysTab<float>&, const RowsDev&, int, double*,
                                            cudaStream_t);
template cudaError_t launch_coherent_amps<double>(const SysTab<double>&, const long long*, const int*,
                                                 int, uint64_t, double*, double*, cudaStream_t);
template cudaError_t launch_init_state<double>(const SysTab<double>&, const double*, const long long*,
                                              const int*, const int2*, int, int, double*, double*, double*,
                                              double*, cudaStream_t);
template cudaError_t launch_step<double>(const SysTab<double>&, const HamDev<double>*, int, int,
                                        const FieldDev<double>*, const int*, const int2*, int,
                                        const int*, int, const double*, const double*, double*, double*, double*,
                                        const double*, int, int, int, int, cudaStream_t);
template cudaError_t launch_gram_integrate<double>(const SysTab<double>&, const double*, const double*,
                                                  const int*, const int2*, int, const int*, int,
                                                  int, double*, cudaStream_t);
template int small_max_configs<double>();
template size_t persistent_smem<double>(long long, int);
template int persistent_ctas<double>(long long, int, int);
template cudaError_t launch_persistent_small<double>(const SysTab<double>&, int, const FieldDev<double>*,
                                                     const double*, const double*, const PItem*, int,
                                                     int*, int, int, uint64_t, double*, int, double*,
                                                     cudaStream_t);
template cudaError_t launch_macro_small<double>(const SysTab<double>&, const HamDev<double>*, int,
                                               const FieldDev<double>*, const int*, const int2*, int,
                                               const int*, int, const double*, double*, double*,
                                               const double*, int, cudaStream_t);
template cudaError_t launch_norm<double>(const SysTab<double>&, const double*, const double*, const int2*,
                                        const int*, int, double*, cudaStream_t);
template cudaError_t launch_trace<double>(const SysTab<double>&, const double*, const int2*, int, int,
                                         const ElecOp&, double*, cudaStream_t);
template cudaError_t launch_finalize<double>(const SysTab<double>&, const RowsDev&, int, double*,
                                            cudaStream_t);

}  // namespace rp
