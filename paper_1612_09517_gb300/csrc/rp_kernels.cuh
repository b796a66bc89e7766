// Device-side data structures and kernel launchers of the radical-pair
// propagation (stochastic trace, Eqs. 13-23 of Lewis, Fay and Manolopoulos).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rp {

constexpr int kMaxNucDev = 24;

// Field-independent Hamiltonian constants in the layout order (rad/us).
// Per nucleus at position p: electron rad[p] (0 or 1), dimension d[p],
// configuration stride stride[p], the 2x2 electron matrix
//   U_p = sum_a u_a S_a,  u_a = (A_ax - i A_ay)/2,
// that multiplies I_+ in S.A.I = sum_a S_a (u_a I_+ + conj(u_a) I_- + A_az I_z),
// stored row-major as (re, im) pairs, and the column (A_xz, A_yz, A_zz).
template <typename T>
struct alignas(16) HamDev {
  long long Z;
  int n_nuc, n_half, n_one, aniso;
  T Je;     // 2J S1.S2 coupling J in rad/us
  T kappa;  // (k_S - k_T)/4: H' = H - i kappa (P_S - P_T)
  int rad[kMaxNucDev];
  int d[kMaxNucDev];
  long long stride[kMaxNucDev];
  T U[kMaxNucDev][8];
  T v[kMaxNucDev][3];
};

// Per-field scalars: Zeeman omega, 1/dE and the shift sh with
// z = (1/dE) H' a - sh a  (sh = E_c/dE for propagation).
template <typename T>
struct FieldDev {
  T omega, s, sh_re, sh_im;
};

enum StepMode { MODE_APPLY = 0, MODE_FIRST = 1, MODE_MID = 2, MODE_LAST = 3 };

// Vector passes (multiples of one state vector of every active row) of the
// Chebyshev term n of a macro-step in the per-term kernels: reads of
// phi_{n-1} (and phi_{n-2}), write of phi_n (not at the last term), the
// accumulator write (first term) or read-modify-write, the singlet slices (a
// quarter each).
inline double term_vector_passes(int n, int n_c) {
  if (n == 1) return 3.5;
  return n == n_c - 1 ? 4.25 : 5.25;
}

// Per-row (one propagation) metadata, device arrays of length rows.  A row is
// active in the macro-steps start <= k < end of its window; rows are refilled
// with new work items as their windows end.
struct RowsDev {
  int* field;        // field index (into the per-field tables)
  int2* win;         // {start, end} macro-step window
  long long* sample; // sample index (coherent) or basis index (deterministic)
  long long* out;    // output slot in the per-sample array
  int* flag;         // rows selected for init / norm / finalize
  double* integral;  // int |P_S psi|^2 dt accumulated (FP64)
  double* survival;  // |psi(T)|^2
};

// Layout description for the state-initialisation kernels.
struct LayoutDev {
  long long Z;
  int n_nuc, n_half, n_one;
  int d[kMaxNucDev];
  int input_index[kMaxNucDev];  // Philox counter word 0 of the nucleus at position p
  long long stride[kMaxNucDev];
};

// Systems of one launch: device arrays of per-system constants, the system of
// each row (NULL: every row is system 0), the slot stride in configurations
// of the row buffers (>= every system's Z), and the Philox pair word of each
// system (pair_of[s], or pair_base + s when pair_of is NULL).
template <typename T>
struct SysTab {
  const HamDev<T>* ham;
  const LayoutDev* lay;
  const double* k_S;
  const int* row_sys;
  long long Zslot;
  uint32_t pair_base;
  const uint32_t* pair_of;
  int* err = nullptr;  // device error word (bit 0: a bounded wait gave up), may be NULL
  // J_z-sector superposition (deterministic = 3): rank of every configuration
  // within its nuclear-M class, and 1/sqrt(n_i) of propagation i (n_i states)
  const int* sec_rank = nullptr;
  const double* sec_scale = nullptr;
};

// ---- launchers (return cudaGetLastError after the launch) ----
// row_flag may be NULL (all rows).  coef holds 4 n_c values per field: the
// Chebyshev coefficients c_n (re, im) in T, then in FP32 the remainders
// c_n - fl(c_n), which the FP32 kernels add so that the coefficients act with
// FP64 accuracy (zero and unused in FP64).

template <typename T>
cudaError_t launch_coherent_amps(const SysTab<T>& S, const long long* row_sample,
                                 const int* row_flag, int rows, uint64_t seed, double* amps,
                                 double* uv, cudaStream_t st);

template <typename T>
cudaError_t launch_init_state(const SysTab<T>& S, const double* amps, const long long* row_sample,
                              const int* row_flag, const int2* row_win, int rows,
                              int deterministic, T* S0, T* S1, double* integral, double* survival,
                              cudaStream_t st);

// One Chebyshev term over every row (see k_cheb_step).  one != NULL: every
// row is that system (its constants travel as kernel parameters); NULL: each
// row reads its system from S.ham.  aniso selects the anisotropic hyperfine
// path (needed if any system of the launch has it).  bulk != 0 allows the FP32
// variant that stages each block's partner tiles with bulk async copies
// (taken for one system with >= 8 spin-1/2 nuclei whose tiles fit in shared
// memory; see k_cheb_step_bulk); its bounded wait reports to S.err.
// macro_dev != NULL: the kernels read the macro-step index from device memory
// (graph replay; see launch_tick), else they use macro.  xblk != 0 writes the
// singlet slices in the tensor-core Gram layout (see launch_gram_tc), else as
// X[row][n][m] complex.
template <typename T>
cudaError_t launch_step(const SysTab<T>& S, const HamDev<T>* one, int aniso, int bulk,
                        const FieldDev<T>* fields, const int* row_field, const int2* row_win,
                        int macro, const int* macro_dev, int rows, const T* cur, const T* prev,
                        T* next, T* acc, T* X, const T* coef, int n_c, int n, int mode,
                        int xblk, cudaStream_t st);

// Largest Z (configurations) that launch_macro_small can hold.
template <typename T>
int small_max_configs();

// A whole macro-step (terms 1 .. n_c - 1) of every active row in one launch,
// one CTA per row with the row's vectors in shared memory (S.Zslot must be
// <= small_max_configs<T>()): reads psi from P, writes the propagated psi to Q
// and the singlet slices to X.
template <typename T>
cudaError_t launch_macro_small(const SysTab<T>& S, const HamDev<T>* one, int aniso,
                               const FieldDev<T>* fields, const int* row_field,
                               const int2* row_win, int macro, const int* macro_dev, int rows,
                               const T* P, T* Q, T* X, const T* coef, int n_c, cudaStream_t st);

// A work item of the persistent launch: field index, system index, macro-steps,
// Philox sample (or basis index) and the slot in the per-sample output.
struct PItem {
  int field, sys, n_macro, pad;
  long long sample, out;
};

// One launch over all n_items work items of small systems (S.Zslot <=
// small_max_configs<T>()): each CTA takes items from *counter (zero before the
// launch) and propagates each item's whole horizon on chip, writing phi_S,
// phi_T and survival to per_sample[3 out ..] (see k_persistent_small).
// Xscratch holds n_c x Zslot complex per CTA; persistent_ctas gives the grid
// (CTAs resident at once; it also sets the kernel's shared-memory attribute,
// so it runs before the launch), persistent_smem the shared memory of a CTA.
template <typename T>
size_t persistent_smem(long long Zs, int n_c);
template <typename T>
int persistent_ctas(long long Zs, int n_c, int aniso);
template <typename T>
cudaError_t launch_persistent_small(const SysTab<T>& S, int aniso, const FieldDev<T>* fields,
                                    const T* coef, const double* W, const PItem* items,
                                    int n_items, int* counter, int n_c, int deterministic,
                                    uint64_t seed, T* Xscratch, int ctas, double* per_sample,
                                    cudaStream_t st);

// A whole macro-step of every active row of one isotropic FP32 system on a
// thread-block cluster per row, the row's Chebyshev vectors in distributed
// shared memory (see k_macro_cluster): reads psi from P, writes the propagated
// psi to Q and the singlet slices to X (tensor-core layout if xblk).
// macro_cluster_plan: whether the system fits (isotropic spin-1/2 and spin-1
// nuclei, Z / 2^c <= 2688 with c <= min(3, n_half)), and the launch shape;
// macro_cluster_max_active:
// clusters of that shape that fit the device at once (0 if none or on error).
struct ClusterPlan {
  int cbits = 0;    // log2 of the CTAs per cluster (per row)
  int local = 0;    // configurations per CTA
  int kpt = 1;      // configurations per thread
  int threads = 0;  // threads per CTA
  size_t smem = 0;  // dynamic shared memory per CTA
};
bool macro_cluster_plan(const HamDev<float>& H, ClusterPlan* out);
// Whether kernel = 0 takes the cluster path: the shapes with a compiled
// instance (measured faster than the per-term kernels).
bool macro_cluster_default(const HamDev<float>& H);
int macro_cluster_max_active(const HamDev<float>& H);
cudaError_t launch_macro_cluster(const HamDev<float>& H, const FieldDev<float>* fields,
                                 const int* row_field, const int2* row_win, int macro,
                                 const int* macro_dev, int rows, const float* P, float* Q,
                                 float* X, const float* coef, int n_c, long long Zslot, int xblk,
                                 cudaStream_t st);

// integral[r] += sum_nm W_nm <x_n|x_m> for the macro-step just finished
// (x_n = singlet slices X[r][n], W per field); one FP64 atomic per CTA.
template <typename T>
cudaError_t launch_gram_integrate(const SysTab<T>& S, const T* X, const double* W,
                                  const int* row_field, const int2* row_win, int macro,
                                  const int* macro_dev, int rows, int n_c, double* integral,
                                  cudaStream_t st);

// The same time integral on the tensor cores (FP32 singlet slices written by
// launch_step with xblk = 1; tcgen05.mma kind::tf32 with a hi/lo split of
// every value, FP64 contraction with W).  Row r covers the configurations of
// its system ham[row_sys[r]] (row_sys NULL: system 0); Zs is the slot stride.
// n_sm sizes the grid; err receives
// bit 0 if a bounded wait gave up.  gram_tc_supported: the accumulator blocks
// of 2 n_c rows fit one 256-column buffer (n_c <= 96).  gram_tc_smem_bytes:
// dynamic shared memory of one CTA.
bool gram_tc_supported(int n_c);
size_t gram_tc_smem_bytes(int n_c);
cudaError_t launch_gram_tc(const float* X, const double* W, const int* row_field,
                           const int2* row_win, int macro, const int* macro_dev, int rows, int n_c,
                           long long Zs, const HamDev<float>* ham, const int* row_sys, int n_sm,
                           double* integral, int* err, cudaStream_t st);

// Floats per row of the singlet slices in the tensor-core Gram layout.
size_t xblk_floats_per_row(long long Zs, int n_c);

// *macro_dev += 1 (one thread): ends a graph-replayed macro-step.
cudaError_t launch_tick(int* macro_dev, cudaStream_t st);

// A 4 x 4 complex operator on the electron states e = 2 e1 + e2 (row-major),
// applied as A x 1 on the nuclei; on = 0 switches it off.
struct ElecOp {
  double re[16], im[16];
  int on;
};

// After macro-step `macro`, for every row active in it (psi = psi(t_i) in Q,
// i = macro + 1 - start): trace[4 i] += |<S|psi>|^2, trace[4 i + 1] += |psi|^2,
// and if A.on trace[4 i + 2] + i trace[4 i + 3] += <psi| A x 1 |psi>.
template <typename T>
cudaError_t launch_trace(const SysTab<T>& S, const T* Q, const int2* row_win, int macro, int rows,
                         const ElecOp& A, double* trace, cudaStream_t st);

template <typename T>
cudaError_t launch_norm(const SysTab<T>& S, const T* S0, const T* S1, const int2* row_win,
                        const int* row_flag, int rows, double* survival, cudaStream_t st);

template <typename T>
cudaError_t launch_finalize(const SysTab<T>& S, const RowsDev& R, int rows, double* per_sample,
                            cudaStream_t st);

// out[f] = (mean phi_S, mean phi_T, SE_S, SE_T, mean survival) over
// per_sample[off[f] .. off[f] + cnt[f]).
cudaError_t launch_stats(const double* per_sample, const long long* off, const long long* cnt,
                         int n_fields, double* out, cudaStream_t st);

// out[f] = (sum_i w_i phi_S, sum_i w_i phi_T, 0, 0, sum_i w_i survival) over
// entry i of per_sample[off[f] .. off[f] + cnt[f]) (w has cnt[f] entries):
// a deterministic trace assembled from weighted propagations.
cudaError_t launch_stats_weighted(const double* per_sample, const long long* off,
                                  const long long* cnt, const double* w, int n_fields,
                                  double* out, cudaStream_t st);

cudaError_t launch_zero(double* p, size_t n, cudaStream_t st);

}  // namespace rp
