// Host-side planning for the Chebyshev propagation of radical-pair wavepackets.
//
// The propagator exp(-iHt - Kt) (Eq. 13) is applied in macro-steps of length h
// with a Chebyshev expansion.  Writing K = kbar/2 + kappa (P_S - P_T) with
// kbar = (k_S + k_T)/2 and kappa = (k_S - k_T)/4 (Eq. 2 with P_S + P_T = 1),
//   exp(-iHt - Kt) = exp(-kbar t / 2) exp(-i H' t),   H' = H - i kappa (P_S - P_T),
// and exp(-i H' tau) = sum_n c_n(tau) T_n((H' - E_c)/dE) with
//   c_n(tau) = (2 - delta_n0) (-i)^n J_n(dE tau) exp(-i E_c tau).
// The singlet probability integrated over one macro-step (Eq. 20 / Eq. 22) is
//   int_0^h |P_S psi(tau)|^2 dtau = sum_nm W_nm <P_S phi_n | P_S phi_m>,
//   W_nm = int_0^h exp(-kbar tau) conj(c_n(tau)) c_m(tau) dtau,
// which this file evaluates by Gauss-Legendre quadrature.
#pragma once

#include <cstdint>

#include <complex>
#include <string>
#include <vector>

namespace rp {

using cplx = std::complex<double>;

// |gamma_e| in rad us^-1 mT^-1 (CODATA 2018).
constexpr double kGammaE = 176.085963023;
constexpr int kMaxNuc = 24;
constexpr int kMaxD = 10;  // 2I + 1 <= 10

// Bessel functions J_0(x) .. J_nmax(x) for x >= 0 by Miller's backward
// recurrence J_{n-1} = (2n/x) J_n - J_{n+1}, normalised with
// J_0 + 2 sum_k J_2k = 1 (Abramowitz and Stegun 9.1.27, 9.1.46).
void bessel_jn(double x, int nmax, double* out);

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_q).
void gauss_legendre(int q, double* x, double* w);

// Smallest and largest eigenvalue of an n x n Hermitian matrix (row-major),
// by cyclic Jacobi rotations on its real symmetric 2n x 2n embedding.
void hermitian_eig_range(int n, const cplx* H, double* lo, double* hi);

// A radical-pair system as the host sees it (energies in rad/us).
struct HostSystem {
  int n_nuc = 0;
  std::vector<int> radical, two_I;   // input order
  std::vector<double> A;             // input order, 9 per nucleus, mT
  double k_S = 0, k_T = 0, J_mT = 0;
  // layout order: order[p] = input index of the nucleus at position p
  std::vector<int> order;
  int n_half = 0, n_one = 0;         // leading spin-1/2 and spin-1 positions
  long long Z = 1;
  std::vector<long long> stride;     // per position
  // per-nucleus hyperfine block S.A.I eigenvalue range (rad/us), per position
  std::vector<double> hf_lo, hf_hi;
  bool aniso = false;
};

struct FieldPlan {
  double E_min = 0, E_max = 0, E_c = 0, dE = 0, h = 0;
  long long n_macro = 0;
  int n_cheb = 0;
  double tail = 0, kbar = 0, kappa = 0, omega = 0;
  std::vector<cplx> coef;  // c_n(h) exp(-kbar h/2), n < n_cheb
  std::vector<cplx> W;     // n_cheb x n_cheb
};

// Fill the derived fields of a HostSystem (layout, strides, hyperfine ranges).
// Returns an empty string on success or an error message.
std::string finish_system(HostSystem& s);

// Plan one field.  Returns an empty string on success or an error message.
std::string plan_field(const HostSystem& s, double B_mT, double t_max, int n_cheb, double tol,
                       bool want_coef, FieldPlan* out);

// Nuclear basis index of sample `sample` for basis-state sampling (Eq. 14
// sampled instead of summed): Philox4x32-10 (Salmon et al., SC'11) with
// counter (0xFFFFFFFF, sample mod 2^32, sample div 2^32, pair) and key
// (seed mod 2^32, seed div 2^32) -- counter word 0 is never a nucleus index,
// so these draws are disjoint from the coherent-state angles -- then
// u = ((x0 >> 5) 2^26 + (x1 >> 6)) / 2^53 and index = min(floor(u Z), Z - 1)
// in FP64.
long long basis_draw(uint64_t seed, uint32_t pair, long long sample, long long Z);

// J_z sectors of the nuclear basis (deterministic = 3): for every
// configuration m (layout order) its rank within the class of configurations
// with the same total nuclear M; n_of[i] = number of classes with more than i
// members, i.e. the states that propagation i carries.  Returns the number of
// propagations (the size of the largest class).
long long sector_table(const HostSystem& hs, std::vector<int>* rank, std::vector<int>* n_of);

// Kernel path rp_yields takes for kernel = 0 on this system in FP32 (5: one
// persistent launch, 2: whole macro-step in one CTA, 4: on a thread-block
// cluster, 1: per-term kernels), and in *cluster_ok whether kernel = 4
// applies to it (rp_api.cu).
int default_kernel_fp32(const HostSystem& hs, bool* cluster_ok);

// Whether kernel = 0 takes the persistent launch for a slot of Zslot
// configurations (<= the one-CTA limit) holding n_systems systems.
bool persistent_default(long long Zslot, int n_systems);

}  // namespace rp
