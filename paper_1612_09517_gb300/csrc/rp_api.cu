// C ABI of the radical-pair stochastic-trace library (declared in include/rp.h).
//
// rp_yields runs, for every (field, sample) pair (a "row"), the macro-step
// Chebyshev propagation of |S> x prod_k |Omega_k> (Eqs. 13, 15, 19) under
// exp(-iHt - Kt) and accumulates k_S int_0^T |P_S psi|^2 dt exactly per
// macro-step (Eqs. 20, 22); rows run concurrently, field-major work items
// sorted by cost, and per-field means and standard errors (Eqs. 18, 23) are
// reduced on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/rp.h"
#include "rp_kernels.cuh"
#include "rp_plan.h"

struct rp_system {
  rp::HostSystem hs;
};

namespace {

thread_local std::string g_err;

rp_alloc_fn g_alloc = nullptr;
rp_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

rp_status fail(rp_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

struct CudaFail {
  rp_status st;
  std::string msg;
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw CudaFail{e == cudaErrorMemoryAllocation ? RP_ENOMEM : RP_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (g_alloc) {
    p = g_alloc(bytes, (void*)st, g_alloc_ctx);
    if (!p) throw CudaFail{RP_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw CudaFail{RP_ENOMEM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
    }
  }
  return p;
}

void dev_free(void* p, cudaStream_t st) {
  if (!p) return;
  if (g_free) g_free(p, (void*)st, g_alloc_ctx);
  else cudaFreeAsync(p, st);
}

// Device allocations released in reverse order when the scope ends.
struct Arena {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Arena(cudaStream_t s) : st(s) {}
  template <typename T>
  T* get(size_t count) {
    void* p = dev_alloc(count * sizeof(T), st);
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Arena() {
    for (auto it = ptrs.rbegin(); it != ptrs.rend(); ++it) dev_free(*it, st);
  }
};

rp_status check_device() {
  static int cached = -1;
  if (cached == 1) return RP_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  cudaDeviceProp prop;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RP_ENODEV, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  if (prop.major != 10 || prop.minor != 3)
    return fail(RP_ENODEV, "this library is built for sm_103a (GB300); device is sm_" +
                               std::to_string(prop.major) + std::to_string(prop.minor));
  cached = 1;
  return RP_OK;
}

template <typename T>
rp::HamDev<T> make_ham(const rp::HostSystem& s) {
  rp::HamDev<T> H;
  std::memset(&H, 0, sizeof(H));
  H.Z = s.Z;
  H.n_nuc = s.n_nuc;
  H.n_half = s.n_half;
  H.n_one = s.n_one;
  H.aniso = s.aniso ? 1 : 0;
  H.Je = (T)(rp::kGammaE * s.J_mT);
  H.kappa = (T)(0.25 * (s.k_S - s.k_T));
  for (int p = 0; p < s.n_nuc; ++p) {
    const int k = s.order[p];
    const double* A = &s.A[9 * k];
    H.rad[p] = s.radical[k];
    H.d[p] = s.two_I[k] + 1;
    H.stride[p] = s.stride[p];
    // u_a = (A_ax - i A_ay)/2 in rad/us; U = sum_a u_a S_a with S = sigma/2
    rp::cplx u[3];
    for (int a = 0; a < 3; ++a)
      u[a] = 0.5 * rp::kGammaE * rp::cplx(A[3 * a + 0], -A[3 * a + 1]);
    const rp::cplx I(0, 1);
    const rp::cplx Um[4] = {0.5 * u[2], 0.5 * (u[0] - I * u[1]), 0.5 * (u[0] + I * u[1]),
                            -0.5 * u[2]};
    for (int i = 0; i < 4; ++i) {
      H.U[p][2 * i] = (T)Um[i].real();
      H.U[p][2 * i + 1] = (T)Um[i].imag();
    }
    for (int a = 0; a < 3; ++a) H.v[p][a] = (T)(rp::kGammaE * A[3 * a + 2]);
  }
  return H;
}

rp::LayoutDev make_layout(const rp::HostSystem& s) {
  rp::LayoutDev L;
  std::memset(&L, 0, sizeof(L));
  L.Z = s.Z;
  L.n_nuc = s.n_nuc;
  L.n_half = s.n_half;
  L.n_one = s.n_one;
  for (int p = 0; p < s.n_nuc; ++p) {
    L.d[p] = s.two_I[s.order[p]] + 1;
    L.input_index[p] = s.order[p];
    L.stride[p] = s.stride[p];
  }
  return L;
}

int default_ncheb(int precision) { return precision == RP_FP64 ? 64 : 88; }
double default_tol(int precision) { return precision == RP_FP64 ? 1e-15 : 1e-9; }

struct Counter {
  long long launches = 0, step_launches = 0;
};

inline void launched(Counter& c, cudaError_t e, const char* what) {
  ck(e, what);
  c.launches++;
}

template <typename T>
rp_status run_yields(rp_system* sys, int n_fields, const double* fields, int M, uint64_t seed,
                     double t_max, const rp_options& o, double* out, double* per_sample,
                     rp_stats* stats) {
  const rp::HostSystem& hs = sys->hs;
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  const double tol = o.tol > 0 ? o.tol : default_tol(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  const long long Mr = o.deterministic ? hs.Z : (long long)M;
  const long long Z = hs.Z;

  // plans per field
  std::vector<rp::FieldPlan> plans(n_fields);
  for (int f = 0; f < n_fields; ++f) {
    std::string e = rp::plan_field(hs, fields[f], t_max, n_c, tol, true, &plans[f]);
    if (!e.empty()) return fail(RP_ENOTCONV, "field " + std::to_string(f) + ": " + e);
  }
  // work items, most expensive field first
  std::vector<int> forder(n_fields);
  for (int f = 0; f < n_fields; ++f) forder[f] = f;
  std::stable_sort(forder.begin(), forder.end(),
                   [&](int a, int b) { return plans[a].n_macro > plans[b].n_macro; });
  const long long items = (long long)n_fields * Mr;

  // rows from the memory budget
  const size_t vec_elems = (size_t)Z * 8;  // T per state vector
  const size_t per_row = (4 * vec_elems + (size_t)n_c * Z * 2) * sizeof(T) +
                         256 + rp::kMaxNucDev * 20 * 8;
  long long rows_cap = o.max_rows > 0 ? o.max_rows : 0;
  if (rows_cap == 0) {
    size_t fr = 0, tot = 0;
    ck(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    const double budget = 0.45 * (double)fr;
    rows_cap = std::max<long long>(1, (long long)(budget / (double)per_row));
  }
  rows_cap = std::min<long long>(rows_cap, 65535);
  const int R = (int)std::min<long long>(items, rows_cap);

  Counter cnt;
  cudaEvent_t ev0, ev1;
  ck(cudaEventCreate(&ev0), "cudaEventCreate");
  ck(cudaEventCreate(&ev1), "cudaEventCreate");
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } evg{ev0, ev1};
  std::vector<cudaEvent_t> pev;  // profiling event pairs
  struct PevGuard {
    std::vector<cudaEvent_t>* v;
    ~PevGuard() {
      for (auto e : *v) cudaEventDestroy(e);
    }
  } pevg{&pev};
  std::vector<double> pev_bytes;
  std::vector<long long> pev_launches;
  ck(cudaEventRecord(ev0, st), "cudaEventRecord");

  long long row_terms = 0;
  double step_bytes_all = 0.0;
  long long h2d = 0, d2h = 0;
  {
    Arena ar(st);
    T* S0 = ar.get<T>((size_t)R * vec_elems);
    T* S1 = ar.get<T>((size_t)R * vec_elems);
    T* F1 = ar.get<T>((size_t)R * vec_elems);
    T* F2 = ar.get<T>((size_t)R * vec_elems);
    T* X = ar.get<T>((size_t)R * n_c * Z * 2);
    double* amps = ar.get<double>((size_t)R * rp::kMaxNucDev * 10 * 2);
    int* d_field = ar.get<int>(R);
    int* d_nmacro = ar.get<int>(R);
    long long* d_sample = ar.get<long long>(R);
    long long* d_out = ar.get<long long>(R);
    double* d_int = ar.get<double>(2 * (size_t)R);
    double* d_surv = d_int + R;
    double* d_ps = ar.get<double>((size_t)items * 3);
    double* d_stats = ar.get<double>((size_t)n_fields * 5);
    rp::FieldDev<T>* d_fdev = ar.get<rp::FieldDev<T>>(n_fields);
    T* d_coef = ar.get<T>((size_t)n_fields * n_c * 2);
    double* d_W = ar.get<double>((size_t)n_fields * n_c * n_c * 2);

    // per-field tables
    std::vector<rp::FieldDev<T>> fdev(n_fields);
    std::vector<T> coef((size_t)n_fields * n_c * 2);
    std::vector<double> W((size_t)n_fields * n_c * n_c * 2);
    for (int f = 0; f < n_fields; ++f) {
      const rp::FieldPlan& P = plans[f];
      fdev[f].omega = (T)P.omega;
      fdev[f].s = (T)(1.0 / P.dE);
      fdev[f].sh_re = (T)(P.E_c / P.dE);
      fdev[f].sh_im = (T)0;
      for (int n = 0; n < n_c; ++n) {
        coef[((size_t)f * n_c + n) * 2] = (T)P.coef[n].real();
        coef[((size_t)f * n_c + n) * 2 + 1] = (T)P.coef[n].imag();
      }
      for (size_t i = 0; i < (size_t)n_c * n_c; ++i) {
        W[((size_t)f * n_c * n_c + i) * 2] = P.W[i].real();
        W[((size_t)f * n_c * n_c + i) * 2 + 1] = P.W[i].imag();
      }
    }
    ck(cudaMemcpyAsync(d_fdev, fdev.data(), fdev.size() * sizeof(fdev[0]), cudaMemcpyHostToDevice, st), "h2d fields");
    ck(cudaMemcpyAsync(d_coef, coef.data(), coef.size() * sizeof(T), cudaMemcpyHostToDevice, st), "h2d coef");
    ck(cudaMemcpyAsync(d_W, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d W");
    h2d += (long long)(fdev.size() * sizeof(fdev[0]) + coef.size() * sizeof(T) + W.size() * sizeof(double));

    const rp::HamDev<T> H = make_ham<T>(hs);
    const rp::LayoutDev L = make_layout(hs);
    const double vbytes = (double)vec_elems * sizeof(T);  // one state vector

    std::vector<int> h_field(R), h_nmacro(R);
    std::vector<long long> h_sample(R), h_out(R);
    for (long long b0 = 0; b0 < items; b0 += R) {
      const int rows = (int)std::min<long long>(R, items - b0);
      long long max_macro = 0;
      std::vector<long long> active_by_macro;
      for (int r = 0; r < rows; ++r) {
        const long long it = b0 + r;
        const int f = forder[it / Mr];
        const long long s = it % Mr;
        h_field[r] = f;
        h_nmacro[r] = (int)plans[f].n_macro;
        h_sample[r] = o.deterministic ? s : o.sample_offset + s;
        h_out[r] = (long long)f * Mr + s;
        max_macro = std::max<long long>(max_macro, plans[f].n_macro);
      }
      active_by_macro.assign(max_macro, 0);
      for (int r = 0; r < rows; ++r)
        for (long long k = 0; k < h_nmacro[r]; ++k) active_by_macro[k]++;
      ck(cudaMemcpyAsync(d_field, h_field.data(), rows * sizeof(int), cudaMemcpyHostToDevice, st), "h2d");
      ck(cudaMemcpyAsync(d_nmacro, h_nmacro.data(), rows * sizeof(int), cudaMemcpyHostToDevice, st), "h2d");
      ck(cudaMemcpyAsync(d_sample, h_sample.data(), rows * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
      ck(cudaMemcpyAsync(d_out, h_out.data(), rows * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
      h2d += (long long)rows * (2 * sizeof(int) + 2 * sizeof(long long));
      launched(cnt, rp::launch_zero(d_int, 2 * (size_t)R, st), "zero integrals");
      if (!o.deterministic)
        launched(cnt, rp::launch_coherent_amps(L, d_sample, rows, seed, o.pair_id, amps, nullptr, st),
                 "coherent amplitudes");
      launched(cnt, rp::launch_init_state<T>(L, amps, d_sample, rows, o.deterministic, S0, st),
               "initial states");

      T* Sb[2] = {S0, S1};
      for (long long k = 0; k < max_macro; ++k) {
        T* P = Sb[k & 1];
        T* Q = Sb[(k + 1) & 1];
        T* phi[3] = {P, F1, F2};
        const long long act = active_by_macro[k];
        const bool prof = o.profile != 0;
        if (prof) {
          cudaEvent_t a, b;
          ck(cudaEventCreate(&a), "cudaEventCreate");
          pev.push_back(a);
          ck(cudaEventCreate(&b), "cudaEventCreate");
          pev.push_back(b);
          ck(cudaEventRecord(a, st), "cudaEventRecord");
        }
        double bytes = 0.0;
        for (int n = 1; n < n_c; ++n) {
          const int mode = (n == 1) ? rp::MODE_FIRST : (n == n_c - 1 ? rp::MODE_LAST : rp::MODE_MID);
          const T* cur = phi[(n - 1) % 3];
          const T* prv = n >= 2 ? phi[(n - 2) % 3] : nullptr;
          T* nxt = phi[n % 3];
          launched(cnt, rp::launch_step<T>(H, d_fdev, d_field, d_nmacro, k, rows, cur, prv,
                                           mode == rp::MODE_LAST ? nullptr : nxt, Q, X, d_coef,
                                           n_c, n, mode, st),
                   "step kernel");
          cnt.step_launches++;
          const double vmul = mode == rp::MODE_FIRST ? 3.5 : (mode == rp::MODE_MID ? 5.25 : 4.25);
          bytes += vmul * vbytes * (double)act;
        }
        if (prof) {
          ck(cudaEventRecord(pev.back(), st), "cudaEventRecord");
          pev_bytes.push_back(bytes);
          pev_launches.push_back(n_c - 1);
        }
        step_bytes_all += bytes;
        row_terms += act * (long long)n_c;
        launched(cnt, rp::launch_gram_integrate<T>(X, d_W, d_field, d_nmacro, k, rows, Z, n_c,
                                                   d_int, st),
                 "gram-integral kernel");
      }
      launched(cnt, rp::launch_norm<T>(S0, S1, d_nmacro, rows, Z, d_surv, st), "norm kernel");
      rp::RowsDev RD{d_field, d_nmacro, d_sample, d_out, d_int, d_surv};
      launched(cnt, rp::launch_finalize(RD, rows, hs.k_S, d_ps, st), "finalize kernel");
    }
    launched(cnt, rp::launch_stats(d_ps, n_fields, Mr, d_stats, st), "stats kernel");
    ck(cudaMemcpyAsync(out, d_stats, (size_t)n_fields * 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h stats");
    d2h += (long long)n_fields * 5 * sizeof(double);
    if (per_sample) {
      ck(cudaMemcpyAsync(per_sample, d_ps, (size_t)items * 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h per-sample");
      d2h += (long long)items * 3 * sizeof(double);
    }
    ck(cudaEventRecord(ev1, st), "cudaEventRecord");
    ck(cudaStreamSynchronize(st), "kernel execution");
  }
  ck(cudaStreamSynchronize(st), "free");
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->kernel_launches = cnt.launches;
    stats->step_launches = cnt.step_launches;
    stats->row_terms = row_terms;
    stats->propagations = items;
    stats->rows = R;
    stats->n_cheb = n_c;
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, ev0, ev1), "cudaEventElapsedTime");
    stats->device_ms = ms;
    double pms = 0.0, pb = 0.0;
    long long pl = 0;
    for (size_t i = 0; i + 1 < pev.size(); i += 2) {
      float t = 0.f;
      ck(cudaEventElapsedTime(&t, pev[i], pev[i + 1]), "cudaEventElapsedTime");
      pms += t;
      pb += pev_bytes[i / 2];
      pl += pev_launches[i / 2];
    }
    stats->step_ms = pms;
    stats->step_bytes = o.profile ? pb : step_bytes_all;
    stats->step_launches_timed = pl;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
  }
  return RP_OK;
}

}  // namespace

namespace rp {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace rp

extern "C" {

const char* rp_version(void) { return "rp-gb300 0.1 (sm_103a)"; }

const char* rp_status_str(rp_status s) {
  switch (s) {
    case RP_OK: return "RP_OK";
    case RP_EINVAL: return "RP_EINVAL";
    case RP_ENOMEM: return "RP_ENOMEM";
    case RP_ECUDA: return "RP_ECUDA";
    case RP_ETIMEOUT: return "RP_ETIMEOUT";
    case RP_ENOTCONV: return "RP_ENOTCONV";
    case RP_ENOTIMPL: return "RP_ENOTIMPL";
    case RP_ENODEV: return "RP_ENODEV";
  }
  return "RP_UNKNOWN";
}

const char* rp_last_error(void) { return g_err.c_str(); }

void rp_default_options(rp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = RP_FP32;
}

rp_status rp_set_allocator(rp_alloc_fn a, rp_free_fn f, void* ctx) {
  if ((a == nullptr) != (f == nullptr)) return fail(RP_EINVAL, "give both allocator hooks or neither");
  g_alloc = a;
  g_free = f;
  g_alloc_ctx = ctx;
  return RP_OK;
}

rp_status rp_create(int n_nuc, const int* radical, const int* two_I, const double* A, double k_S,
                    double k_T, double J, rp_system** out) {
  g_err.clear();
  if (!out) return fail(RP_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_nuc < 0 || n_nuc > rp::kMaxNuc) return fail(RP_EINVAL, "n_nuc must be in [0, 24]");
  if (n_nuc > 0 && (!radical || !two_I || !A)) return fail(RP_EINVAL, "NULL nucleus array");
  if (!std::isfinite(k_S) || !std::isfinite(k_T) || k_S < 0 || k_T < 0)
    return fail(RP_EINVAL, "rates must be finite and >= 0");
  if (k_S == 0 && k_T == 0) return fail(RP_EINVAL, "k_S and k_T cannot both be 0");
  if (!std::isfinite(J)) return fail(RP_EINVAL, "J must be finite");
  rp_system* s = new (std::nothrow) rp_system;
  if (!s) return fail(RP_ENOMEM, "host allocation failed");
  rp::HostSystem& h = s->hs;
  h.n_nuc = n_nuc;
  h.k_S = k_S;
  h.k_T = k_T;
  h.J_mT = J;
  for (int k = 0; k < n_nuc; ++k) {
    if (radical[k] != 0 && radical[k] != 1) {
      delete s;
      return fail(RP_EINVAL, "radical[" + std::to_string(k) + "] must be 0 or 1");
    }
    if (two_I[k] < 1 || two_I[k] > 9) {
      delete s;
      return fail(RP_EINVAL, "two_I[" + std::to_string(k) + "] must be in [1, 9]");
    }
    const double* a = A + 9 * k;
    double sc = 0.0;
    for (int i = 0; i < 9; ++i) {
      if (!std::isfinite(a[i])) {
        delete s;
        return fail(RP_EINVAL, "non-finite hyperfine tensor entry");
      }
      sc = std::max(sc, std::fabs(a[i]));
    }
    for (int i = 0; i < 3; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (std::fabs(a[3 * i + j] - a[3 * j + i]) > 1e-12 * std::max(sc, 1e-300)) {
          delete s;
          return fail(RP_EINVAL, "hyperfine tensor " + std::to_string(k) + " is not symmetric");
        }
    h.radical.push_back(radical[k]);
    h.two_I.push_back(two_I[k]);
    for (int i = 0; i < 9; ++i) h.A.push_back(a[i]);
  }
  std::string e = rp::finish_system(h);
  if (!e.empty()) {
    delete s;
    return fail(RP_EINVAL, e);
  }
  *out = s;
  return RP_OK;
}

void rp_destroy(rp_system* s) { delete s; }

rp_status rp_layout(const rp_system* s, int* order, long long* Z_out) {
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (order)
    for (int p = 0; p < s->hs.n_nuc; ++p) order[p] = s->hs.order[p];
  if (Z_out) *Z_out = s->hs.Z;
  return RP_OK;
}

rp_status rp_plan_field(const rp_system* s, double B, double t_max, int precision, int n_cheb,
                        double tol, rp_field_plan* plan, double* coef, double* W) {
  if (!s || !plan) return fail(RP_EINVAL, "NULL argument");
  if (precision != RP_FP64 && precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  const int n_c = n_cheb > 0 ? n_cheb : default_ncheb(precision);
  const double tl = tol > 0 ? tol : default_tol(precision);
  rp::FieldPlan P;
  std::string e = rp::plan_field(s->hs, B, t_max, n_c, tl, coef || W, &P);
  if (!e.empty()) return fail(RP_ENOTCONV, e);
  plan->E_min = P.E_min;
  plan->E_max = P.E_max;
  plan->E_c = P.E_c;
  plan->dE = P.dE;
  plan->h = P.h;
  plan->n_macro = P.n_macro;
  plan->n_cheb = P.n_cheb;
  plan->tail = P.tail;
  plan->kbar = P.kbar;
  plan->kappa = P.kappa;
  if (coef)
    for (int n = 0; n < n_c; ++n) {
      coef[2 * n] = P.coef[n].real();
      coef[2 * n + 1] = P.coef[n].imag();
    }
  if (W)
    for (size_t i = 0; i < (size_t)n_c * n_c; ++i) {
      W[2 * i] = P.W[i].real();
      W[2 * i + 1] = P.W[i].imag();
    }
  return RP_OK;
}

rp_status rp_yields(rp_system* s, int n_fields, const double* fields, int M, uint64_t seed,
                    double t_max, const rp_options* opt, double* out, double* per_sample,
                    rp_stats* stats) {
  g_err.clear();
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (n_fields < 0) return fail(RP_EINVAL, "n_fields must be >= 0");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (!o.deterministic && M < 2) return fail(RP_EINVAL, "M must be >= 2 (the standard error needs it)");
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return fail(RP_EINVAL, "t_max must be positive and finite");
  if (o.sample_offset < 0) return fail(RP_EINVAL, "sample_offset must be >= 0");
  if (n_fields > 0 && (!fields || !out)) return fail(RP_EINVAL, "NULL fields or out");
  for (int f = 0; f < n_fields; ++f)
    if (!std::isfinite(fields[f])) return fail(RP_EINVAL, "non-finite field");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_fields == 0) return RP_OK;
  rp_status ds = check_device();
  if (ds != RP_OK) return ds;
  try {
    if (o.precision == RP_FP64)
      return run_yields<double>(s, n_fields, fields, M, seed, t_max, o, out, per_sample, stats);
    return run_yields<float>(s, n_fields, fields, M, seed, t_max, o, out, per_sample, stats);
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
}

rp_status rp_apply_h(rp_system* s, double B, int precision, int n_vec, const void* x, void* y,
                     void* stream) {
  g_err.clear();
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (precision != RP_FP64 && precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (n_vec < 0 || n_vec > 65535) return fail(RP_EINVAL, "n_vec must be in [0, 65535]");
  if (!std::isfinite(B)) return fail(RP_EINVAL, "field must be finite");
  if (n_vec == 0) return RP_OK;
  if (!x || !y || x == y) return fail(RP_EINVAL, "x and y must be distinct device arrays");
  rp_status ds = check_device();
  if (ds != RP_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  const rp::HostSystem& hs = s->hs;
  try {
    Arena ar(st);
    const double kbar = 0.5 * (hs.k_S + hs.k_T);
    if (precision == RP_FP64) {
      rp::FieldDev<double> F{rp::kGammaE * B, 1.0, 0.0, 0.5 * kbar};
      auto* d = ar.get<rp::FieldDev<double>>(1);
      ck(cudaMemcpyAsync(d, &F, sizeof(F), cudaMemcpyHostToDevice, st), "h2d");
      ck(rp::launch_step<double>(make_ham<double>(hs), d, nullptr, nullptr, 0, n_vec,
                                 (const double*)x, nullptr, (double*)y, nullptr, nullptr, nullptr,
                                 0, 0, rp::MODE_APPLY, st), "apply kernel");
    } else {
      rp::FieldDev<float> F{(float)(rp::kGammaE * B), 1.f, 0.f, (float)(0.5 * kbar)};
      auto* d = ar.get<rp::FieldDev<float>>(1);
      ck(cudaMemcpyAsync(d, &F, sizeof(F), cudaMemcpyHostToDevice, st), "h2d");
      ck(rp::launch_step<float>(make_ham<float>(hs), d, nullptr, nullptr, 0, n_vec,
                                (const float*)x, nullptr, (float*)y, nullptr, nullptr, nullptr, 0,
                                0, rp::MODE_APPLY, st), "apply kernel");
    }
    ck(cudaStreamSynchronize(st), "apply kernel execution");
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  }
  return RP_OK;
}

rp_status rp_init_states(rp_system* s, int precision, uint64_t seed, uint32_t pair_id,
                         long long sample0, int n, void* psi, double* angles, void* stream) {
  g_err.clear();
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (precision != RP_FP64 && precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (n < 0 || n > 65535) return fail(RP_EINVAL, "n must be in [0, 65535]");
  if (sample0 < 0) return fail(RP_EINVAL, "sample0 must be >= 0");
  if (n == 0) return RP_OK;
  if (!psi) return fail(RP_EINVAL, "psi is NULL");
  rp_status ds = check_device();
  if (ds != RP_OK) return ds;
  cudaStream_t st = (cudaStream_t)stream;
  const rp::HostSystem& hs = s->hs;
  try {
    Arena ar(st);
    std::vector<long long> smp(n);
    for (int i = 0; i < n; ++i) smp[i] = sample0 + i;
    long long* d_s = ar.get<long long>(n);
    double* amps = ar.get<double>((size_t)n * rp::kMaxNucDev * 10 * 2);
    double* uv = angles ? ar.get<double>((size_t)n * std::max(hs.n_nuc, 1) * 2) : nullptr;
    ck(cudaMemcpyAsync(d_s, smp.data(), n * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    const rp::LayoutDev L = make_layout(hs);
    ck(rp::launch_coherent_amps(L, d_s, n, seed, pair_id, amps, uv, st), "coherent amplitudes");
    if (precision == RP_FP64)
      ck(rp::launch_init_state<double>(L, amps, d_s, n, 0, (double*)psi, st), "initial states");
    else
      ck(rp::launch_init_state<float>(L, amps, d_s, n, 0, (float*)psi, st), "initial states");
    if (angles && hs.n_nuc > 0)
      ck(cudaMemcpyAsync(angles, uv, (size_t)n * hs.n_nuc * 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "init kernels");
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  }
  return RP_OK;
}

}  // extern "C"
