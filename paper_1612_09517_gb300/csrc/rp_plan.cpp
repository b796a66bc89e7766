// Host-side planning: spectral bounds, Chebyshev coefficients and time-integral
// weights for the macro-step propagation (see rp_plan.h for the formulas).
#include "rp_plan.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <string>

namespace rp {

void bessel_jn(double x, int nmax, double* out) {
  for (int k = 0; k <= nmax; ++k) out[k] = 0.0;
  if (x == 0.0) {
    out[0] = 1.0;
    return;
  }
  const int big = std::max(nmax, static_cast<int>(x));
  int m = big + 32 + static_cast<int>(std::sqrt(40.0 * (big + 1)));
  m += (m & 1);  // start from an even order
  std::vector<double> v(nmax + 1, 0.0);
  double jp1 = 0.0;  // J_{n+1}
  double jn = 1e-30; // J_n, arbitrary seed at n = m
  double norm = 2.0 * jn;  // m is even and > 0
  for (int n = m; n >= 1; --n) {
    const double jm1 = (2.0 * n / x) * jn - jp1;
    jp1 = jn;
    jn = jm1;  // now J_{n-1}
    const int k = n - 1;
    if (k <= nmax) v[k] = jn;
    if (k == 0) norm += jn;
    else if ((k & 1) == 0) norm += 2.0 * jn;
    if (std::fabs(jn) > 1e200) {  // rescale to stay in range
      jn *= 1e-200;
      jp1 *= 1e-200;
      norm *= 1e-200;
      for (int i = k; i <= nmax; ++i) v[i] *= 1e-200;
    }
  }
  for (int k = 0; k <= nmax; ++k) out[k] = v[k] / norm;
}

void gauss_legendre(int q, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (q + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (q + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_q(z), p0 = P_{q-1}(z)
      dp = q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = q * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = -z;
    x[q - 1 - i] = z;
    w[i] = w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  if (q == 1) {
    x[0] = 0.0;
    w[0] = 2.0;
  }
}

void hermitian_eig_range(int n, const cplx* H, double* lo, double* hi) {
  // Real symmetric embedding [[Re, -Im], [Im, Re]]: each eigenvalue twice.
  const int N = 2 * n;
  std::vector<double> a(N * N);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const cplx h = H[i * n + j];
      a[i * N + j] = h.real();
      a[(i + n) * N + (j + n)] = h.real();
      a[i * N + (j + n)] = -h.imag();
      a[(i + n) * N + j] = h.imag();
    }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, scale = 0.0;
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        if (i != j) off += a[i * N + j] * a[i * N + j];
        scale += a[i * N + j] * a[i * N + j];
      }
    if (off <= 1e-30 * (scale + 1e-300)) break;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        const double apq = a[p * N + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * N + q] - a[p * N + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) /
                         (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < N; ++k) {  // rotate columns p, q
          const double akp = a[k * N + p], akq = a[k * N + q];
          a[k * N + p] = c * akp - s * akq;
          a[k * N + q] = s * akp + c * akq;
        }
        for (int k = 0; k < N; ++k) {  // rotate rows p, q
          const double apk = a[p * N + k], aqk = a[q * N + k];
          a[p * N + k] = c * apk - s * aqk;
          a[q * N + k] = s * apk + c * aqk;
        }
      }
  }
  double l = a[0], h = a[0];
  for (int i = 1; i < N; ++i) {
    l = std::min(l, a[i * N + i]);
    h = std::max(h, a[i * N + i]);
  }
  *lo = l;
  *hi = h;
}

namespace {

// Spin operators of spin I = two_I/2 in the basis j = 0..2I (M = I - j).
void spin_ops(int two_I, std::vector<cplx>& Ix, std::vector<cplx>& Iy, std::vector<cplx>& Iz) {
  const int d = two_I + 1;
  const double I = 0.5 * two_I;
  Ix.assign(d * d, 0.0);
  Iy.assign(d * d, 0.0);
  Iz.assign(d * d, 0.0);
  for (int j = 0; j < d; ++j) Iz[j * d + j] = I - j;
  for (int j = 1; j < d; ++j) {
    const double M = I - j;  // <j-1| I_+ |j> = sqrt(I(I+1) - M(M+1))
    const double c = std::sqrt(I * (I + 1) - M * (M + 1));
    // I_x = (I_+ + I_-)/2, I_y = (I_+ - I_-)/(2i)
    Ix[(j - 1) * d + j] += 0.5 * c;
    Ix[j * d + (j - 1)] += 0.5 * c;
    Iy[(j - 1) * d + j] += cplx(0.0, -0.5 * c);
    Iy[j * d + (j - 1)] += cplx(0.0, 0.5 * c);
  }
}

}  // namespace

std::string finish_system(HostSystem& s) {
  const int n = s.n_nuc;
  s.order.resize(n);
  std::iota(s.order.begin(), s.order.end(), 0);
  std::stable_sort(s.order.begin(), s.order.end(),
                   [&](int a, int b) { return s.two_I[a] < s.two_I[b]; });
  s.n_half = s.n_one = 0;
  for (int p = 0; p < n; ++p) {
    if (s.two_I[s.order[p]] == 1) s.n_half++;
    else if (s.two_I[s.order[p]] == 2) s.n_one++;
  }
  s.stride.resize(n);
  long long Z = 1;
  for (int p = 0; p < n; ++p) {
    s.stride[p] = Z;
    Z *= (s.two_I[s.order[p]] + 1);
    if (Z > (1LL << 31)) return "Z = prod(2I+1) exceeds 2^31";
  }
  s.Z = Z;
  s.aniso = false;
  for (int k = 0; k < n; ++k) {
    const double* A = &s.A[9 * k];
    const double sc = std::max({std::fabs(A[0]), std::fabs(A[4]), std::fabs(A[8]), 1e-300});
    if (std::fabs(A[1]) > 0 || std::fabs(A[2]) > 0 || std::fabs(A[5]) > 0 ||
        std::fabs(A[0] - A[4]) > 1e-15 * sc || std::fabs(A[0] - A[8]) > 1e-15 * sc)
      s.aniso = true;
  }
  // hyperfine block sum_ab A_ab S_a (x) I_b, electron index major
  s.hf_lo.assign(n, 0.0);
  s.hf_hi.assign(n, 0.0);
  std::vector<cplx> Sx, Sy, Sz;
  spin_ops(1, Sx, Sy, Sz);
  const std::vector<cplx>* S[3] = {&Sx, &Sy, &Sz};
  for (int p = 0; p < n; ++p) {
    const int k = s.order[p];
    const int d = s.two_I[k] + 1;
    std::vector<cplx> Ix, Iy, Iz;
    spin_ops(s.two_I[k], Ix, Iy, Iz);
    const std::vector<cplx>* I[3] = {&Ix, &Iy, &Iz};
    const int D = 2 * d;
    std::vector<cplx> h(D * D, 0.0);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double Aab = kGammaE * s.A[9 * k + 3 * a + b];
        if (Aab == 0.0) continue;
        for (int e = 0; e < 2; ++e)
          for (int f = 0; f < 2; ++f)
            for (int i = 0; i < d; ++i)
              for (int j = 0; j < d; ++j)
                h[(e * d + i) * D + (f * d + j)] += Aab * (*S[a])[e * 2 + f] * (*I[b])[i * d + j];
      }
    hermitian_eig_range(D, h.data(), &s.hf_lo[p], &s.hf_hi[p]);
  }
  return "";
}

namespace {

// Bernstein-ellipse parameter rho of the smallest ellipse with foci +-1
// containing the rectangle [-1, 1] x [-delta, delta].
double ellipse_rho(double delta) {
  if (delta <= 0.0) return 1.0;
  double lo = 1.0, hi = 2.0 + 4.0 * std::sqrt(delta) + 2.0 * delta;
  for (int it = 0; it < 200; ++it) {
    const double r = 0.5 * (lo + hi);
    const double a = 0.5 * (r + 1.0 / r), b = 0.5 * (r - 1.0 / r);
    if (1.0 / (a * a) + delta * delta / (b * b) <= 1.0) hi = r;
    else lo = r;
  }
  return hi;
}

double tail_bound(double x, int n_c, double rho, double crouzeix) {
  const int extra = 120;
  std::vector<double> J(n_c + extra + 1);
  bessel_jn(x, n_c + extra, J.data());
  double t = 0.0, rp = std::pow(rho, n_c);
  for (int n = n_c; n <= n_c + extra; ++n) {
    t += 2.0 * std::fabs(J[n]) * rp;
    rp *= rho;
  }
  return crouzeix * t;
}

}  // namespace

std::string plan_field(const HostSystem& s, double B_mT, double t_max, int n_c, double tol,
                       bool want_coef, FieldPlan* out) {
  if (n_c < 8 || n_c > 256) return "n_cheb must be in [8, 256]";
  if (!(tol > 0.0 && tol < 1e-2)) return "tol must be in (0, 1e-2)";
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return "t_max must be positive and finite";
  if (!std::isfinite(B_mT)) return "field must be finite";
  FieldPlan& P = *out;
  const double omega = kGammaE * B_mT;
  const double Je = kGammaE * s.J_mT;
  // Hermitian electron block omega (S1z + S2z) + 2J S1.S2: eigenvalues
  // omega + J/2 (T+), J/2 (T0), -omega + J/2 (T-), -3J/2 (S)
  const double ev[4] = {omega + 0.5 * Je, 0.5 * Je, -omega + 0.5 * Je, -1.5 * Je};
  double lo = *std::min_element(ev, ev + 4), hi = *std::max_element(ev, ev + 4);
  for (int p = 0; p < s.n_nuc; ++p) {  // Weyl: lambda(A + B) within [lo_A + lo_B, hi_A + hi_B]
    lo += s.hf_lo[p];
    hi += s.hf_hi[p];
  }
  P.E_min = lo;
  P.E_max = hi;
  P.E_c = 0.5 * (hi + lo);
  P.dE = 0.5 * (hi - lo) * (1.0 + 1e-12) + 1e-12 * (std::fabs(hi) + std::fabs(lo)) + 1e-9;
  P.kbar = 0.5 * (s.k_S + s.k_T);
  P.kappa = 0.25 * (s.k_S - s.k_T);
  P.omega = omega;
  P.n_cheb = n_c;
  const double delta = std::fabs(P.kappa) / P.dE;
  const double rho = ellipse_rho(delta);
  const double crz = delta > 0.0 ? 1.0 + std::sqrt(2.0) : 1.0;  // Crouzeix's constant
  // largest x = dE h with the truncation bound below tol
  double xl = 0.0, xh = static_cast<double>(n_c);
  if (tail_bound(1e-6, n_c, rho, crz) > tol) return "tolerance unreachable with this n_cheb";
  for (int it = 0; it < 100; ++it) {
    const double xm = 0.5 * (xl + xh);
    if (tail_bound(xm, n_c, rho, crz) <= tol) xl = xm;
    else xh = xm;
  }
  const double h_max = xl / P.dE;
  const double nm = std::ceil(t_max / h_max);
  if (!(nm >= 1.0) || nm > 4e9) return "too many macro-steps for t_max";
  P.n_macro = static_cast<long long>(nm);
  P.h = t_max / static_cast<double>(P.n_macro);
  const double x = P.dE * P.h;
  P.tail = tail_bound(x, n_c, rho, crz);
  if (!want_coef) return "";
  // propagation coefficients c_n(h) with the factored decay exp(-kbar h/2)
  std::vector<double> J(n_c + 1);
  bessel_jn(x, n_c, J.data());
  P.coef.resize(n_c);
  const cplx phase = std::exp(cplx(-0.5 * P.kbar * P.h, -P.E_c * P.h));
  const cplx mi(0.0, -1.0);
  cplx ipow(1.0, 0.0);  // (-i)^n
  for (int n = 0; n < n_c; ++n) {
    P.coef[n] = phase * ipow * ((n == 0 ? 1.0 : 2.0) * J[n]);
    ipow *= mi;
  }
  // W_nm = eps_n eps_m i^(n-m) int_0^h exp(-kbar tau) J_n(dE tau) J_m(dE tau) dtau
  const int q = n_c + static_cast<int>(std::ceil(x)) + 48;
  std::vector<double> gx(q), gw(q), Jq((size_t)q * (n_c + 1));
  gauss_legendre(q, gx.data(), gw.data());
  for (int i = 0; i < q; ++i) {
    const double tau = 0.5 * P.h * (gx[i] + 1.0);
    bessel_jn(P.dE * tau, n_c, &Jq[(size_t)i * (n_c + 1)]);
    gw[i] *= 0.5 * P.h * std::exp(-P.kbar * tau);
  }
  P.W.assign((size_t)n_c * n_c, 0.0);
  const cplx ipw[4] = {cplx(1, 0), cplx(0, 1), cplx(-1, 0), cplx(0, -1)};  // i^k
  for (int n = 0; n < n_c; ++n)
    for (int m = n; m < n_c; ++m) {
      double acc = 0.0;
      for (int i = 0; i < q; ++i)
        acc += gw[i] * Jq[(size_t)i * (n_c + 1) + n] * Jq[(size_t)i * (n_c + 1) + m];
      const double eps = (n == 0 ? 1.0 : 2.0) * (m == 0 ? 1.0 : 2.0);
      const cplx v = eps * acc * ipw[((n - m) % 4 + 4) % 4];
      P.W[(size_t)n * n_c + m] = v;
      P.W[(size_t)m * n_c + n] = std::conj(v);
    }
  return "";
}

namespace {

// One Philox4x32-10 block (ten rounds; multipliers and Weyl key increments of
// the published generator).
void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

}  // namespace

long long basis_draw(uint64_t seed, uint32_t pair, long long sample, long long Z) {
  uint32_t c[4] = {0xFFFFFFFFu, (uint32_t)((uint64_t)sample & 0xFFFFFFFFu),
                   (uint32_t)((uint64_t)sample >> 32), pair};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
  const double u = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) *
                   (1.0 / 9007199254740992.0);
  long long idx = (long long)std::floor(u * (double)Z);
  if (idx > Z - 1) idx = Z - 1;
  return idx;
}

long long sector_table(const HostSystem& hs, std::vector<int>* rank, std::vector<int>* n_of) {
  // twice the nuclear M of configuration m: sum_p (2 I_p - 2 j_p) with digit
  // j_p = I_p - M_p of position p (the layout's digits count down from +I_p)
  int two_max = 0;
  for (int p = 0; p < hs.n_nuc; ++p) two_max += hs.two_I[hs.order[p]];
  std::vector<long long> count(2 * (size_t)two_max + 1, 0);
  rank->assign((size_t)hs.Z, 0);
  for (long long m = 0; m < hs.Z; ++m) {
    int two_M = 0;
    for (int p = 0; p < hs.n_nuc; ++p) {
      const int d = hs.two_I[hs.order[p]] + 1;
      const long long j = (m / hs.stride[p]) % d;
      two_M += (d - 1) - 2 * (int)j;
    }
    long long& c_ = count[(size_t)(two_M + two_max)];
    (*rank)[(size_t)m] = (int)c_;
    ++c_;
  }
  long long n_prop = 0;
  for (long long c_ : count) n_prop = std::max(n_prop, c_);
  n_of->assign((size_t)n_prop, 0);
  for (long long c_ : count)
    for (long long i = 0; i < c_; ++i) (*n_of)[(size_t)i]++;
  return n_prop;
}

}  // namespace rp
