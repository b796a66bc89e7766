/*
 * rp.h -- C ABI of the GB300 library for the stochastic spin-coherent-state
 * trace of radical-pair recombination yields (Lewis, Fay and Manolopoulos,
 * "An efficient quantum mechanical method for radical pair recombination
 * reactions").
 *
 * Model (Sec. II):
 *   H   = omega (S_1z + S_2z) + 2 J S_1.S_2 + sum_k S_{i(k)} . A_k . I_k     (Eq. 1)
 *         omega = |gamma_e| B with B along z; the paper's isotropic coupling
 *         a_ik I.S is the special case A_k = a_k 1.
 *   K   = k_S/2 P_S + k_T/2 P_T                                               (Eq. 2)
 *   P_S = 1/4 - S_1.S_2,   P_T = 3/4 + S_1.S_2                                (Eqs. 3-4)
 *   |S, Omega; t> = exp(-iHt - Kt) |S> x prod_k |Omega_k>                   (Eqs. 13, 15, 19)
 *   phi_S(Omega) = k_S int_0^T <S,Omega;t| P_S |S,Omega;t> dt                 (Eq. 22, truncated at T)
 *   Phi_S(B) ~ (1/M) sum_s phi_S(Omega_s),  SE = sigma / sqrt(M)              (Eqs. 18, 20, 23)
 * The triplet yield is Phi_T = 1 - survival(T) - Phi_S, which follows from
 * d|psi|^2/dt = -k_S <P_S> - k_T <P_T> for the Haberkorn generator (Eq. 2).
 *
 * Units: fields, hyperfine tensors and J in mT; rates in us^-1; times in us.
 * Internally energies are in rad/us (value in mT times |gamma_e|).
 *
 * Conventions for every entry point:
 *   - Host pointers are caller-owned; they are read or written during the
 *     call only and never retained.  Device pointers (named *_dev) must be
 *     CUDA device memory on the current device.
 *   - Every function returns an rp_status; no C++ exception crosses the ABI.
 *     On failure, rp_last_error() returns a thread-local message.
 *   - An rp_system is owned by the library from rp_create to rp_destroy.
 *     Calls on one system are not thread-safe.
 *   - Compute entry points run on the CUDA stream given in rp_options.stream
 *     (or the legacy default stream when NULL) and synchronise that
 *     stream before returning, so host outputs are complete on return.
 *
 * State vector layout (rp_apply_h, rp_init_states): complex interleaved
 * (re, im) in double (RP_FP64) or float (RP_FP32).  Element (m, e) of vector
 * v is at complex index v * 4Z + 4 m + e, where e = 2 e_1 + e_2 with
 * e_i = 0 for alpha (m_s = +1/2) and 1 for beta, and m = sum_p j_p stride_p
 * is the nuclear configuration in the library's nucleus order (see
 * rp_layout): position p = 0 is the innermost nucleus, stride_0 = 1,
 * stride_{p+1} = stride_p (2 I_p + 1), and digit j_p = I_p - M_p counts down
 * from M_p = +I_p.
 */
#ifndef RP_H_
#define RP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rp_system rp_system; /* opaque, library-owned */

typedef enum rp_status {
  RP_OK = 0,
  RP_EINVAL = 1,    /* invalid argument (message in rp_last_error) */
  RP_ENOMEM = 2,    /* device or host allocation failed */
  RP_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed */
  RP_ETIMEOUT = 4,  /* a bounded device wait gave up */
  RP_ENOTCONV = 5,  /* the propagation plan could not reach the tolerance */
  RP_ENOTIMPL = 6,  /* option combination not implemented */
  RP_ENODEV = 7     /* no usable CUDA device (sm_103a) */
} rp_status;

enum { RP_FP64 = 0, RP_FP32 = 1 };

/* Options of the compute entry points.  rp_default_options fills defaults. */
typedef struct rp_options {
  int precision;          /* RP_FP64 or RP_FP32: storage and arithmetic of the
                             state vectors; time integrals, Chebyshev
                             coefficients and averages are FP64 always */
  int n_cheb;             /* Chebyshev terms per macro-step, multiple of 4 in [8, 88]
                             (0: 88) */
  double tol;             /* truncation bound per macro-step (0: 1e-15 FP64, 1e-9 FP32) */
  int max_rows;           /* concurrent propagations (0: from free device memory) */
  int deterministic;      /* 1: trace over the Z basis states |S, M> (Eq. 14)
                             instead of M coherent-state samples; M is ignored.
                             2: M basis states |S, M> drawn uniformly at random
                             (rp_basis_indices) instead of coherent states, an
                             unbiased estimate of the same trace (rp_yields and
                             rp_time_trace only);
                             3: the trace of Eq. 14 regrouped by J_z sector
                             (rp_yields, isotropic systems): propagation i
                             carries the normalised sum of the i-th basis state
                             |S, m> of every class of nuclear configurations
                             with the same total M.  H, K and P_S conserve J_z
                             (field along z, isotropic couplings), so the
                             cross terms between classes vanish and the
                             propagation's yield is the mean of its n_i states';
                             the trace is sum_i (n_i / Z) phi_i over the
                             largest class's size of propagations
                             (rp_trace_propagations) instead of Z */
  long long sample_offset;/* first sample index (resume / sharding) */
  uint32_t pair_id;       /* Philox counter word 3 (radical-pair id) */
  int profile;            /* 1: time the H.psi step kernels with CUDA events */
  void* stream;           /* cudaStream_t, NULL: the legacy default stream */
  int kernel;             /* 0: choose (5 where 128 <= Z <= 1024, or a batch of
                             several systems fits one CTA, and graph = 0; 2
                             where Z fits one CTA's shared memory otherwise; 4
                             for the FP32 shapes with a compiled cluster
                             instance -- 8 spin-1/2 and 4 spin-1 nuclei,
                             isotropic, one system; else 1);
                             1: one launch per Chebyshev term (any Z);
                             2: a whole macro-step per launch with each row's
                             vectors in shared memory (Z <= 2048 FP32, 1024
                             FP64; larger Z falls back to 1); 3: as 1, and FP32
                             single systems with >= 8 spin-1/2 nuclei stage
                             each block's partner configurations with bulk
                             async copies (slower than 1 on the workloads
                             measured so far; a candidate of rp_tune);
                             4: a whole macro-step per launch on a cluster of
                             2^c CTAs per row (c <= 3) holding the row's
                             Chebyshev vectors in distributed shared memory
                             (FP32, one isotropic system with Z / 2^c <= 2688,
                             2^c <= 2^(number of spin-1/2 nuclei); otherwise
                             falls back to 1);
                             5: one persistent launch over all propagations of
                             the call: each CTA takes (field, sample) items
                             from a device counter and runs an item's whole
                             horizon with its vectors in shared memory (the
                             time integral on CUDA cores in the same CTA);
                             Z <= 2048 FP32, 1024 FP64, deterministic 0-2,
                             rp_yields, rp_yields_batch and the converged
                             entries; elsewhere kernel 5 selects as 0 */
  int gram;               /* time integral (Eqs. 20, 22) of each macro-step: 0 choose
                             (2 where it applies); 1 CUDA cores (any precision);
                             2 tensor cores (FP32 single systems with the
                             per-term kernels: tcgen05.mma
                             kind::tf32 on hi/lo-split values, FP32 partial
                             sums, FP64 contraction; otherwise falls back to 1) */
  int graph;              /* 1: capture each macro-step's launches (Chebyshev terms
                             and time integral) in a CUDA graph and replay it; the
                             kernels then read the macro-step index from a device
                             counter.  Refill work between macro-steps stays eager.
                             Results are identical to graph = 0. */
} rp_options;

/* Per-call statistics (optional output of rp_yields). */
typedef struct rp_stats {
  long long kernel_launches;    /* kernels launched by the call */
  long long step_launches;      /* of which H.psi Chebyshev step kernels */
  long long row_terms;          /* sum over propagations of Chebyshev terms */
  long long propagations;       /* (field, sample) propagations run */
  double step_bytes;            /* algorithmic bytes of the timed step launches */
  double step_ms;               /* CUDA-event time of the timed step launches (profile=1) */
  long long step_launches_timed;/* step launches inside the timed intervals */
  double device_ms;             /* CUDA-event time of the whole call on its stream */
  int rows;                     /* concurrent propagations used */
  int n_cheb;                   /* Chebyshev terms per macro-step used */
  long long h2d_bytes;          /* host-to-device bytes copied by the call */
  long long d2h_bytes;          /* device-to-host bytes copied by the call */
  long long graph_launches;     /* macro-steps replayed from a CUDA graph (graph = 1);
                                   their kernels are counted in kernel_launches */
  int kernel_path;              /* kernel path of the Chebyshev terms (rp_options.kernel
                                   values 1-5; rp_yields and rp_yields_converged) */
  double cv_ms;                 /* rp_yields_cv: host wall time of the control-variate
                                   work (training, mu = E[g], evaluation, estimates) */
} rp_stats;

/* Propagation plan of one field (rp_plan_field; host logic, no GPU needed). */
typedef struct rp_field_plan {
  double E_min, E_max;   /* rigorous bounds on the spectrum of H (rad/us) */
  double E_c, dE;        /* Chebyshev centre and half-width (rad/us) */
  double h;              /* macro-step length (us) */
  long long n_macro;     /* macro-steps to reach t_max */
  int n_cheb;            /* terms per macro-step */
  double tail;           /* truncation bound of the plan */
  double kbar;           /* (k_S + k_T)/2, factored out of the propagator */
  double kappa;          /* (k_S - k_T)/4, remaining non-Hermitian part */
} rp_field_plan;

/* Device allocator hooks: alloc(bytes, stream, ctx) -> device pointer or
 * NULL; free(ptr, stream, ctx).  NULL restores cudaMallocAsync/cudaFreeAsync. */
typedef void* (*rp_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*rp_free_fn)(void* ptr, void* stream, void* ctx);

/* Library version string. */
const char* rp_version(void);

/* Human-readable name of a status code (static storage). */
const char* rp_status_str(rp_status s);

/* Thread-local message of the last failure in this thread ("" if none). */
const char* rp_last_error(void);

/* Fill *opt with defaults: RP_FP32, n_cheb 0, tol 0, max_rows 0,
 * deterministic 0, sample_offset 0, pair_id 0, profile 0, stream NULL,
 * kernel 0. */
void rp_default_options(rp_options* opt);

/* Route the library's device allocations through the caller's allocator
 * (e.g. a framework's caching allocator).  Process-wide. */
rp_status rp_set_allocator(rp_alloc_fn alloc, rp_free_fn free_fn, void* ctx);

/* Create a radical-pair system (Eq. 1 with Eqs. 2-4).
 *   n_nuc     number of nuclei, 0 <= n_nuc <= 24
 *   radical   [n_nuc] 0 or 1: the electron each nucleus couples to
 *   two_I     [n_nuc] twice the nuclear spin, 1 <= two_I <= 9
 *   A         [n_nuc * 9] hyperfine tensors in mT, row-major 3x3, symmetric
 *             to 1e-12 relative (the isotropic a_k of Eq. 1 is a_k * identity)
 *   k_S, k_T  recombination rates (us^-1), finite, >= 0, not both 0 (Eq. 2)
 *   J         exchange coupling in mT, entering as +2J S_1.S_2 (Eq. 1)
 * Z = prod(2 I_k + 1) must not exceed 2^31.  Host-only: needs no GPU.
 * Errors: RP_EINVAL on any violated condition, RP_ENOMEM. */
rp_status rp_create(int n_nuc, const int* radical, const int* two_I, const double* A,
                    double k_S, double k_T, double J, rp_system** out);

/* Release a system (NULL is ignored). */
void rp_destroy(rp_system* sys);

/* The same radical pair with the field along the unit vector
 * n(theta, phi) = (sin theta cos phi, sin theta sin phi, cos theta) instead of
 * z (Eq. 1 with omega = |gamma_e| B n): a new system whose hyperfine tensors
 * are R A_k R^T with R = R_y(-theta) R_z(-phi), the rotation that takes n to z
 * (isotropic tensors are unchanged).  Yields and traces of the new system at
 * field B are those of the original with the field B n; the coherent-state
 * directions it samples are drawn in the rotated frame (the lab direction of
 * a sample direction n_k is R^T n_k).  Host-only.  Errors: RP_EINVAL, RP_ENOMEM. */
rp_status rp_rotate(const rp_system* sys, double theta, double phi, rp_system** out);

/* Nucleus order of the state layout: order[p] = input index of the nucleus at
 * position p (p = 0 innermost); *Z_out = number of nuclear states.  Either
 * output may be NULL. */
rp_status rp_layout(const rp_system* sys, int* order, long long* Z_out);

/* Host planner for field B (mT) and horizon t_max (us): spectral bounds of H
 * by Weyl's inequality over the electron block and each hyperfine block, the
 * Chebyshev centre and half-width, and the macro-step h chosen so that the
 * truncated series stays below tol.  Optionally returns the n_cheb
 * propagation coefficients c_n (complex, 2 doubles each; they include the
 * factored decay exp(-kbar h / 2)) and the n_cheb x n_cheb time-integral
 * weights W_nm (complex, row-major) of one macro-step.  Host-only.
 * precision/n_cheb/tol as in rp_options (0 = defaults).
 * Errors: RP_EINVAL, RP_ENOTCONV. */
rp_status rp_plan_field(const rp_system* sys, double B, double t_max, int precision,
                        int n_cheb, double tol, rp_field_plan* plan,
                        double* coef, double* W);

/* Singlet and triplet yields over a field sweep (Eqs. 18, 20, 22, 23).
 *   fields      [n_fields] field strengths B in mT (n_fields >= 0; 0 is a no-op)
 *   M           coherent-state samples per field, >= 2 (ignored when
 *               opt->deterministic, which uses the Z basis states |S, M>)
 *   seed        Philox key; sample s of nucleus k draws counter
 *               (k, s_lo, s_hi, pair_id) with key (seed_lo, seed_hi)
 *   t_max       horizon T > 0 (us)
 *   opt         NULL for defaults
 *   out         [n_fields * 5] host: Phi_S, Phi_T, SE_S, SE_T, mean survival
 *               (deterministic = 3: the trace, SE 0)
 *   per_sample  [n_fields * M * 3] host or NULL: phi_S, phi_T, survival of
 *               each (field, sample), field-major (M = rp_trace_propagations
 *               when deterministic is 1 or 3)
 *   stats       optional host output
 * Every sample uses the same directions at every field (common random numbers).
 * Errors: RP_EINVAL, RP_ENOMEM, RP_ECUDA, RP_ENOTCONV, RP_ENODEV. */
rp_status rp_yields(rp_system* sys, int n_fields, const double* fields, int M, uint64_t seed,
                    double t_max, const rp_options* opt, double* out, double* per_sample,
                    rp_stats* stats);

/* Yields over a field sweep to a target standard error (Eq. 23) at every field
 * (the "SE <= target on the whole curve" criterion; Eqs. 18, 20, 22).
 * Each field first gets M_min coherent-state samples; then, in rounds, each
 * field whose standard error of Phi_S is above se_target gets the samples its
 * measured spread asks for, ceil(1.15 sigma_f^2 / se_target^2) + 1, at most 4x
 * its samples so far per round, capped at M_max.  Sample s uses the same directions at every field.  All rounds run
 * on one pool of rows that are refilled as propagations finish.
 *   out     [n_fields * 5] host: Phi_S, Phi_T, SE_S, SE_T, mean survival
 *   M_used  [n_fields] host or NULL: samples used per field
 * opt->deterministic must be 0.  Errors as rp_yields. */
rp_status rp_yields_converged(rp_system* sys, int n_fields, const double* fields, double se_target,
                              int M_min, int M_max, uint64_t seed, double t_max,
                              const rp_options* opt, double* out, int* M_used, rp_stats* stats);

/* Yields of several radical pairs of uneven size in one call (the same
 * quantities as rp_yields for each pair).  System s has n_fields[s] fields
 * fields[s], M[s] >= 2 samples per field and horizon t_max[s]; it draws its
 * directions with Philox pair word opt->pair_id + s, so its results equal
 * those of rp_yields on that system with pair_id + s.  Systems are grouped by
 * size (a row slot holds at most twice a system's Z) and each group runs all
 * its (system, field, sample) propagations on one pool of rows that is
 * refilled as propagations finish.
 *   out[s]  [n_fields[s] * 5] host: Phi_S, Phi_T, SE_S, SE_T, mean survival
 * opt->deterministic must be 0.  Errors as rp_yields. */
rp_status rp_yields_batch(int n_sys, rp_system* const* systems, const int* n_fields,
                          const double* const* fields, const int* M, const double* t_max,
                          uint64_t seed, const rp_options* opt, double* const* out,
                          rp_stats* stats);

/* y = (H - iK) x for n_vec state vectors in the layout above, field B (mT);
 * x_dev and y_dev are device arrays of n_vec * 4Z complex values in the
 * precision given, and must not overlap.  Stream as in rp_options (may be
 * NULL).  Errors: RP_EINVAL, RP_ECUDA. */
rp_status rp_apply_h(rp_system* sys, double B, int precision, int n_vec, const void* x_dev,
                     void* y_dev, void* stream);

/* Initial states |S> x prod_k |Omega_k> (Eqs. 15, 19) of samples
 * sample0 .. sample0 + n - 1 written to psi_dev (n * 4Z complex, precision as
 * given).  angles, if not NULL, receives [n * n_nuc * 2] host doubles: the
 * uniforms (u1, u2) of each nucleus in input order, with cos(theta) = 1 - 2 u1
 * and phi = 2 pi u2.  Errors: RP_EINVAL, RP_ECUDA, RP_ENODEV. */
rp_status rp_init_states(rp_system* sys, int precision, uint64_t seed, uint32_t pair_id,
                         long long sample0, int n, void* psi_dev, double* angles, void* stream);

/* ---- learned control variate (Eqs. 18, 23 with a control variate) ----
 * g(Omega, B): a multilayer perceptron (SiLU hidden layers, linear output,
 * BF16 weights, FP32 activations and accumulation) of 3 n_nuc + 10 features:
 * n(Omega_k) for every nucleus k in input order (Eq. 16); the classical
 * hyperfine fields b_r = sum_{k on radical r} I_k A_k n(Omega_k) / B_hyp,r
 * (B_hyp of Eq. 21, a_k^2 generalised to |A_k|_F^2 / 3); |b_1|, |b_2|,
 * b_1 . b_2; B / B_scale -- with Omega_k drawn by the same Philox map as
 * rp_yields.  Trained by mean
 * squared error on per-sample yields; the estimate of one field is
 * Phi_cv = mean(phi - beta (g - mu)), beta = cov(phi, g)/var(g), mu = E[g].
 * Training must use samples disjoint from those of the estimate. */
typedef struct rp_cv rp_cv; /* opaque, library-owned */

typedef struct rp_cv_options {
  int hidden;            /* hidden width (default 256) */
  int layers;            /* hidden layers (default 3) */
  int epochs;            /* training epochs (default 200) */
  int batch;             /* minibatch size (default 256) */
  double lr;             /* Adam learning rate (default 1e-3) */
  double weight_decay;   /* decoupled weight decay (default 1e-4) */
  double B_scale;        /* field scale of the last feature, mT (default 10) */
  uint64_t init_seed;    /* weight initialisation and shuffling seed (default 1) */
  void* stream;          /* cudaStream_t, NULL: the legacy default stream */
} rp_cv_options;

/* Defaults above. */
void rp_cv_default_options(rp_cv_options* opt);

/* Network for the nuclei of sys (input dimension 3 n_nuc + 10), initialised
 * uniformly with scale sqrt(6 / fan_in) (hidden) and sqrt(3 / fan_in) (output),
 * zero biases.  Errors: RP_EINVAL, RP_ENOMEM, RP_ECUDA, RP_ENODEV. */
rp_status rp_cv_create(const rp_system* sys, const rp_cv_options* opt, rp_cv** out);

/* Release a network (NULL is ignored). */
void rp_cv_destroy(rp_cv* cv);

/* Copy the flat FP32 parameter vector (W_0, b_0, W_1, b_1, ...; W_l row-major
 * (out, in)) out to get and/or in from set (host arrays of *count floats);
 * *count receives the number of parameters.  Setting refreshes the BF16
 * weights. */
rp_status rp_cv_params(rp_cv* cv, float* get, const float* set, long long* count);

/* Loss 1/(2n) sum (g(x_i) - y_i)^2 and its gradient for n host feature rows
 * x (n x (3 n_nuc + 10), FP32) and targets y; grad has *count floats. */
rp_status rp_cv_loss_grad(rp_cv* cv, int n, const float* x, const float* y, double* loss,
                          float* grad);

/* Train on n per-sample yields phi of samples[i] at fields B[i] (mT) drawn with
 * (seed, pair_id); targets are phi standardised per distinct field.  Adam,
 * shuffled minibatches; loss_per_epoch (host, epochs doubles) may be NULL. */
rp_status rp_cv_train(rp_cv* cv, int n, const double* B, const long long* samples, uint64_t seed,
                      uint32_t pair_id, const double* phi, double* loss_per_epoch);

/* g at n (field, sample) pairs; g is a host array of n doubles. */
rp_status rp_cv_eval(rp_cv* cv, int n, const double* B, const long long* samples, uint64_t seed,
                     uint32_t pair_id, double* g);

/* mu_f = mean of g over samples 0 .. n_mc-1 of (seed, pair_id) at each field,
 * and var_mu_f = var(g) / n_mc (host arrays of n_fields doubles). */
rp_status rp_cv_mean(rp_cv* cv, int n_fields, const double* B, long long n_mc, uint64_t seed,
                     uint32_t pair_id, double* mu, double* var_mu);

/* Per-field control-variate estimates from per-sample yields (rp_yields
 * layout: phi_S, phi_T, survival triples) and g of the same samples, field f
 * owning entries [offsets[f], offsets[f] + counts[f]) (counts >= 2).
 * out [n_fields * 5]: Phi_cv, SE_cv, Phi_plain, SE_plain, beta, where
 * SE_cv^2 = var(phi - beta g)/M + beta^2 var_mu (Eq. 23). */
rp_status rp_cv_estimate(rp_cv* cv, int n_fields, const long long* offsets, const long long* counts,
                         const double* per_sample, const double* g, const double* mu,
                         const double* var_mu, double* out);

/* Plan of rp_yields_cv. */
typedef struct rp_cv_plan {
  int M_train;        /* plain samples per control-variate field, used for training (default 300) */
  int cv_threshold;   /* a field whose plain estimate would need at least this many
                         samples uses the control variate (default 150) */
  long long n_mc;     /* directions per field for mu = E[g] (default 2^18) */
  rp_cv_options net;  /* network and training options (rp_cv_default_options) */
} rp_cv_plan;

/* Defaults above. */
void rp_cv_default_plan(rp_cv_plan* plan);

/* Singlet yields over a field sweep to a target standard error at every field,
 * with the learned control variate where it pays (Eqs. 18, 20, 22, 23):
 *  1. M_min plain samples (indices sample_offset + 0, 1, ...) at every field;
 *     fields whose plain estimate would need fewer than
 *     max(cv_threshold, 2 M_train) samples continue with plain rounds as
 *     rp_yields_converged does (each round at most 4x the samples so far);
 *  2. the other fields get plain samples up to M_train; one network is trained
 *     on all of them (rp_cv_train) and mu = E[g] is computed per field from
 *     n_mc directions of a separate stream (pair word with bit 30 set);
 *  3. those fields then draw fresh samples (indices from 2^40 + sample_offset,
 *     disjoint from the training samples, so the estimate stays unbiased),
 *     estimate with the control variate (rp_cv_estimate) and combine it with
 *     their plain estimate by inverse-variance weights until the combined SE
 *     reaches se_target (or M_max samples).
 *   out [n_fields * 8]: Phi_S, SE_S (combined), Phi_S and SE of the plain
 *     samples, Phi_S and SE of the control-variate samples, beta, 1 if the
 *     field used the control variate else 0
 *   M_plain, M_cv [n_fields] host or NULL: samples of each kind per field
 * opt->deterministic must be 0; sample_offset < 2^39.  Errors as rp_yields. */
rp_status rp_yields_cv(rp_system* sys, int n_fields, const double* fields, double se_target,
                       int M_min, int M_max, uint64_t seed, double t_max, const rp_options* opt,
                       const rp_cv_plan* plan, double* out, int* M_plain, int* M_cv,
                       rp_stats* stats);

/* rp_yields without device allocation.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory while
 * they run -- e.g. a host application that hands each plug-in a fixed
 * device-memory budget and forbids calls to the allocator, or a long-running
 * service that must not fail part-way because an allocation failed.
 * Arguments, outputs and errors are those of rp_yields.  All device scratch
 * (state vectors, singlet slices, Gram matrices, per-row bookkeeping,
 * per-field tables, per-sample results) comes from one file-scope device array
 * of 64 MiB (67108864 bytes) that every GPU loading the library holds until
 * the process exits; no cudaMalloc/cudaFree or allocating routine is called.
 * Rows are batched to fit the array; a workload whose fixed part plus one row
 * does not fit is rejected with RP_EINVAL and a message giving the bytes it
 * needs.  All calls share the array and find the previous call's contents in
 * it (the call clears what must start at zero); calls that overlap on the GPU
 * race on it.  The first call on a device looks up the array's address with
 * that device current and should come before any stream capture; the
 * address is kept for the life of the process, so after a cudaDeviceReset of
 * that device this entry point must not be called there again.
 * rp_stats.device_ms and the step timings are not measured (0).
 * It always runs the per-term kernels (kernel = 1) with the CUDA-core time
 * integral (gram = 1), eagerly: kernel and gram other than 0 or 1, graph
 * other than 0, and opt->deterministic = 2 (random basis states) are refused
 * with RP_ENOTIMPL; max_rows > 0 caps the rows of a batch. */
rp_status rp_yields_static(rp_system* sys, int n_fields, const double* fields, int M,
                           uint64_t seed, double t_max, const rp_options* opt, double* out,
                           double* per_sample, rp_stats* stats);

/* Time-resolved observables of one field (Eq. 18 with A = P_S, P_T and the
 * identity; Eqs. 3-4): the sample means of
 *   P_S(t) = |<S|psi(t)>|^2,  P_T(t) = |psi(t)|^2 - P_S(t),  survival |psi(t)|^2
 * at the macro-step boundaries t_i = i h, i = 0 .. n_macro (h from
 * rp_plan_field), over M coherent-state samples (or the Z basis states of
 * Eq. 14 when opt->deterministic).  psi(0) = |S> x nuclear state, so the first
 * point is (1, 0, 1).  The same propagation as rp_yields; graph replay is not
 * used.
 *   max_times  capacity of t and out (in time points)
 *   n_times    [out] n_macro + 1
 *   t          [n_times] host, us;  out [n_times * 3] host: P_S, P_T, survival
 * With t or out NULL only *n_times is set (a size query).
 * Errors: RP_EINVAL (max_times < n_times, M < 1, bad options), RP_ENOTCONV,
 * RP_ECUDA, RP_ENOMEM, RP_ENODEV. */
/* Basis indices drawn by deterministic = 2 for samples sample_offset ..
 * sample_offset + M - 1 (host only): Philox4x32-10 with counter
 * (0xFFFFFFFF, s mod 2^32, s div 2^32, pair_id) and key (seed mod 2^32,
 * seed div 2^32); u = ((x0 >> 5) 2^26 + (x1 >> 6)) / 2^53 and
 * index = min(floor(u Z), Z - 1) in FP64.  out [M] host.  Errors: RP_EINVAL. */
rp_status rp_basis_indices(uint64_t seed, uint32_t pair_id, long long sample_offset, int M,
                           long long Z, long long* out);

rp_status rp_time_trace(rp_system* sys, double B, int M, uint64_t seed, double t_max,
                        const rp_options* opt, int max_times, int* n_times, double* t,
                        double* out);

/* Time-resolved expectation of an electron operator (Eq. 18 with A = A_e x 1
 * on the nuclei; Eqs. 7-9): the sample mean of <psi(t)| A_e x 1 |psi(t)> at
 * the macro-step boundaries of one field, with psi(t) the decaying wavepacket
 * of Eq. 13 (so, as for P_S(t) in rp_time_trace, recombined population no
 * longer contributes).  A_e is 4 x 4 complex, row-major, 32 doubles (re, im),
 * in the electron basis e = 2 e_1 + e_2 (alpha = 0, beta = 1).
 *   t    [n_times] host, us;  out [n_times * 2] host: Re, Im of the mean
 * Other arguments, the size query and errors as rp_time_trace. */
rp_status rp_time_observable(rp_system* sys, double B, int M, uint64_t seed, double t_max,
                             const rp_options* opt, const double* A_e, int max_times,
                             int* n_times, double* t, double* out);

/* Combining estimates over disjoint sample sets (Eqs. 18, 23; host only), for
 * sharding the samples over processes: rp_field_sums turns an rp_yields output
 * block over M >= 2 samples (n_fields x 5: Phi_S, Phi_T, SE_S, SE_T, mean
 * survival) into the per-field sums (sum phi_S, sum phi_S^2, sum phi_T,
 * sum phi_T^2, sum survival), exactly up to rounding; rp_combine_sums turns
 * sums added over sample sets with M samples in all back into an output
 * block (M - 1 in the sample variance).  Errors: RP_EINVAL. */
rp_status rp_field_sums(int n_fields, const double* out, long long M, double* sums);
rp_status rp_combine_sums(int n_fields, const double* sums, long long M, double* out);

/* Propagations per field of a deterministic trace (host only): Z for
 * deterministic = 1 (Eq. 14), the size of the largest class of nuclear
 * configurations with equal total M for deterministic = 3 (the J_z-sector
 * regrouping; isotropic systems only).  rp_yields with these modes writes
 * that many per-sample entries per field.  Errors: RP_EINVAL, RP_ENOMEM. */
rp_status rp_trace_propagations(const rp_system* sys, int deterministic, long long* n);

/* Launch-configuration autotuner (the paper has no counterpart: its method
 * ran serially on CPUs).  For one system, precision and concurrency it times
 * the candidates
 *   kernel in {1, 2 (only if Z fits in shared memory), 3 (only FP32 with
 *   >= 8 spin-1/2 nuclei, where it stages partner tiles)},
 *   n_cheb in {32, 48, 64, 88},  graph in {0, 1}
 * on `rows` coherent-state samples at field B (mT) over six macro-steps
 * through rp_yields (one untimed run, the faster of two timed runs by the
 * call's CUDA events) and keeps the one with the most propagated
 * sample-microseconds per second.  Every candidate meets the same truncation
 * tolerance, so the choice changes speed, not results beyond rounding.
 *   base   options to start from (NULL: defaults); precision, tol, stream and
 *          deterministic are kept, kernel/n_cheb/graph are chosen and
 *          max_rows is set to rows
 *   tuned  [out] base with the chosen settings
 *   res    [out, may be NULL] the choice, its rate, the rate of base's own
 *          settings (-1 if base's settings were not a candidate) and the
 *          number of candidates timed
 * If the environment variable RP_TUNE_CACHE names a file, results are looked
 * up there first (key: device name and SM count, precision, sorted spins,
 * anisotropy, Z, rows, |B| to 3 digits, deterministic) and new results are
 * appended; a hit times nothing (res->from_cache = 1).
 * Errors: RP_EINVAL (rows < 2, bad precision, non-finite B, NULL), plus any
 * error of rp_plan_field / rp_yields. */
typedef struct rp_tune_result {
  int kernel, n_cheb, graph;
  double rate;       /* propagated sample-us per second of device time */
  double base_rate;  /* same for base's own settings, -1 if not timed */
  int candidates;    /* candidates timed (0 on a cache hit) */
  int from_cache;
} rp_tune_result;

rp_status rp_tune(rp_system* sys, double B, int rows, const rp_options* base,
                  rp_options* tuned, rp_tune_result* res);

#ifdef __cplusplus
}
#endif

#endif /* RP_H_ */
