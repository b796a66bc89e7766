// rp_yields_static: the field-sweep yields of rp_yields with every piece of
// device scratch taken from one fixed, file-scope device array instead of
// device allocations.
//
// Who needs it: callers that must not allocate device memory at run time --
// for example a host application that gives each plug-in a fixed device-memory
// budget and forbids it from calling the allocator, or a long-running service
// that must not fail halfway through a run because an allocation failed.  They
// pass host inputs and outputs as for rp_yields; all work buffers (state
// vectors, singlet slices, Gram matrices, per-row bookkeeping, per-field
// tables, per-sample results) live in g_rp_static_scratch.
//
// Limits and sharing: the array holds kStaticScratchBytes (64 MiB) on every
// GPU that loads the library, until the process exits.  Rows are batched so
// that one batch fits; a call whose fixed part plus a single row does not fit
// is rejected with RP_EINVAL.  Every call on a device reuses the same array and
// finds the previous call's contents there; the code clears what must start
// at zero.  Calls that overlap on the GPU (other streams, other host threads)
// race on the array.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress, with that device current); that first call
// should come before any stream capture.  The address is kept for the life of
// the process: a caller that resets the device (cudaDeviceReset) must not call
// this entry point on that device afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/rp.h"
#include "rp_kernels.cuh"
#include "rp_plan.h"

struct rp_system {
  rp::HostSystem hs;
};

namespace rp {
void set_last_error(const std::string& msg);  // rp_api.cu: message of rp_last_error()
}

namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;

static __device__ __align__(256) unsigned char g_rp_static_scratch[kStaticScratchBytes];

rp_status sfail(rp_status s, const std::string& m) {
  rp::set_last_error(m);
  return s;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_addr_mu;
std::vector<void*> g_addr;

rp_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(RP_ENODEV, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rp_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return sfail(RP_ECUDA, std::string("cudaGetSymbolAddress(g_rp_static_scratch): ") +
                                 cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[dev]);
  return RP_OK;
}

struct StaticFail {
  rp_status st;
  std::string msg;
};

void sck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw StaticFail{RP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Bump allocation inside the scratch array.
struct Bump {
  unsigned char* base;
  size_t used = 0;
  template <typename T>
  T* get(size_t count) {
    T* p = reinterpret_cast<T*>(base + used);
    used += up256(count * sizeof(T));
    return p;
  }
};

template <typename T>
rp::HamDev<T> ham_of(const rp::HostSystem& s) {
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
    rp::cplx u[3];
    for (int a = 0; a < 3; ++a) u[a] = 0.5 * rp::kGammaE * rp::cplx(A[3 * a + 0], -A[3 * a + 1]);
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

rp::LayoutDev layout_of(const rp::HostSystem& s) {
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

template <typename T>
rp_status run_static(const rp::HostSystem& hs, int n_fields, const double* fields, int M,
                     uint64_t seed, double t_max, const rp_options& o, double* out,
                     double* per_sample, rp_stats* stats, unsigned char* scratch) {
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : 88;
  const double tol = o.tol > 0 ? o.tol : (o.precision == RP_FP64 ? 1e-15 : 1e-9);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return sfail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  const long long Mr = o.deterministic ? hs.Z : (long long)M;
  const long long Z = hs.Z;
  std::vector<rp::FieldPlan> plans(n_fields);
  for (int f = 0; f < n_fields; ++f) {
    std::string e = rp::plan_field(hs, fields[f], t_max, n_c, tol, true, &plans[f]);
    if (!e.empty()) return sfail(RP_ENOTCONV, "field " + std::to_string(f) + ": " + e);
  }
  std::vector<int> forder(n_fields);
  for (int f = 0; f < n_fields; ++f) forder[f] = f;
  std::stable_sort(forder.begin(), forder.end(),
                   [&](int a, int b) { return plans[a].n_macro > plans[b].n_macro; });
  const long long items = (long long)n_fields * Mr;

  // scratch budget: fixed per-call part plus rows
  const size_t vec = (size_t)Z * 8;
  const size_t fixed = up256((size_t)items * 3 * sizeof(double)) + up256((size_t)n_fields * 5 * sizeof(double)) +
                       up256(2 * (size_t)n_fields * sizeof(long long)) +
                       up256(sizeof(rp::HamDev<T>)) + up256(sizeof(rp::LayoutDev)) + up256(sizeof(double)) +
                       up256((size_t)n_fields * sizeof(rp::FieldDev<T>)) +
                       up256((size_t)n_fields * n_c * 4 * sizeof(T)) +
                       up256((size_t)n_fields * n_c * n_c * 2 * sizeof(double));
  auto rows_bytes = [&](size_t R) {
    return 4 * up256(R * vec * sizeof(T)) + up256(R * n_c * Z * 2 * sizeof(T)) +
           up256(R * rp::kMaxNucDev * 20 * sizeof(double)) + up256(R * sizeof(int)) +
           up256(R * sizeof(int2)) + 2 * up256(R * sizeof(long long)) + up256(2 * R * sizeof(double));
  };
  if (fixed + rows_bytes(1) > kStaticScratchBytes)
    return sfail(RP_EINVAL, "rp_yields_static needs " + std::to_string(fixed + rows_bytes(1)) +
                                " bytes of scratch for this workload; the static array holds " +
                                std::to_string(kStaticScratchBytes) + " bytes");
  size_t R = 1;
  const size_t R_cap = o.max_rows > 0 ? std::min<size_t>((size_t)o.max_rows, 65535) : 65535;
  while (R < (size_t)items && R < R_cap && fixed + rows_bytes(R + 1) <= kStaticScratchBytes) ++R;

  Bump b{scratch};
  double* d_ps = b.get<double>((size_t)items * 3);
  double* d_stats = b.get<double>((size_t)n_fields * 5);
  long long* d_offcnt = b.get<long long>(2 * (size_t)n_fields);
  auto* d_fdev = b.get<rp::FieldDev<T>>(n_fields);
  T* d_coef = b.get<T>((size_t)n_fields * n_c * 4);
  double* d_W = b.get<double>((size_t)n_fields * n_c * n_c * 2);
  T* S0 = b.get<T>(R * vec);
  T* S1 = b.get<T>(R * vec);
  T* F1 = b.get<T>(R * vec);
  T* F2 = b.get<T>(R * vec);
  T* X = b.get<T>(R * n_c * Z * 2);
  double* amps = b.get<double>(R * rp::kMaxNucDev * 20);
  int* d_field = b.get<int>(R);
  int2* d_win = b.get<int2>(R);
  long long* d_sample = b.get<long long>(R);
  long long* d_out = b.get<long long>(R);
  double* d_int = b.get<double>(2 * R);
  double* d_surv = d_int + R;

  std::vector<rp::FieldDev<T>> fdev(n_fields);
  std::vector<T> coef((size_t)n_fields * n_c * 4, T(0));  // c_n, then (FP32) c_n - fl(c_n)
  std::vector<double> W((size_t)n_fields * n_c * n_c * 2);
  for (int f = 0; f < n_fields; ++f) {
    const rp::FieldPlan& P = plans[f];
    fdev[f].omega = (T)P.omega;
    fdev[f].s = (T)(1.0 / P.dE);
    fdev[f].sh_re = (T)(P.E_c / P.dE);
    fdev[f].sh_im = (T)0;
    for (int n = 0; n < n_c; ++n) {
      const T re = (T)P.coef[n].real(), im = (T)P.coef[n].imag();
      T* cf = &coef[(size_t)f * n_c * 4];
      cf[2 * n] = re;
      cf[2 * n + 1] = im;
      if (sizeof(T) == 4) {
        cf[2 * n_c + 2 * n] = (T)(P.coef[n].real() - (double)re);
        cf[2 * n_c + 2 * n + 1] = (T)(P.coef[n].imag() - (double)im);
      }
    }
    for (size_t i = 0; i < (size_t)n_c * n_c; ++i) {
      W[((size_t)f * n_c * n_c + i) * 2] = P.W[i].real();
      W[((size_t)f * n_c * n_c + i) * 2 + 1] = P.W[i].imag();
    }
  }
  long long launches = 0, steps = 0, row_terms = 0, h2d = 0, d2h = 0;
  auto L1 = [&](cudaError_t e, const char* w) {
    sck(e, w);
    launches++;
  };
  sck(cudaMemcpyAsync(d_fdev, fdev.data(), fdev.size() * sizeof(fdev[0]), cudaMemcpyHostToDevice, st), "h2d");
  sck(cudaMemcpyAsync(d_coef, coef.data(), coef.size() * sizeof(T), cudaMemcpyHostToDevice, st), "h2d");
  sck(cudaMemcpyAsync(d_W, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
  h2d += (long long)(fdev.size() * sizeof(fdev[0]) + coef.size() * sizeof(T) + W.size() * sizeof(double));

  const rp::HamDev<T> H = ham_of<T>(hs);
  const rp::LayoutDev L = layout_of(hs);
  auto* d_ham = b.get<rp::HamDev<T>>(1);
  auto* d_lay = b.get<rp::LayoutDev>(1);
  double* d_kS = b.get<double>(1);
  sck(cudaMemcpyAsync(d_ham, &H, sizeof(H), cudaMemcpyHostToDevice, st), "h2d");
  sck(cudaMemcpyAsync(d_lay, &L, sizeof(L), cudaMemcpyHostToDevice, st), "h2d");
  sck(cudaMemcpyAsync(d_kS, &hs.k_S, sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
  h2d += (long long)(sizeof(H) + sizeof(L) + sizeof(double));
  const rp::SysTab<T> SYS{d_ham, d_lay, d_kS, nullptr, Z, o.pair_id, nullptr};
  std::vector<int> h_field(R);
  std::vector<int2> h_win(R);
  std::vector<long long> h_sample(R), h_out(R);
  for (long long b0 = 0; b0 < items; b0 += (long long)R) {
    const int rows = (int)std::min<long long>((long long)R, items - b0);
    long long max_macro = 0;
    for (int r = 0; r < rows; ++r) {
      const long long it = b0 + r;
      const int f = forder[it / Mr];
      const long long s = it % Mr;
      h_field[r] = f;
      h_win[r] = make_int2(0, (int)plans[f].n_macro);
      h_sample[r] = o.deterministic ? s : o.sample_offset + s;
      h_out[r] = (long long)f * Mr + s;
      max_macro = std::max<long long>(max_macro, plans[f].n_macro);
    }
    sck(cudaMemcpyAsync(d_field, h_field.data(), rows * sizeof(int), cudaMemcpyHostToDevice, st), "h2d");
    sck(cudaMemcpyAsync(d_win, h_win.data(), rows * sizeof(int2), cudaMemcpyHostToDevice, st), "h2d");
    sck(cudaMemcpyAsync(d_sample, h_sample.data(), rows * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    sck(cudaMemcpyAsync(d_out, h_out.data(), rows * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    h2d += (long long)rows * (sizeof(int) + sizeof(int2) + 2 * sizeof(long long));
    // the array keeps the previous call's contents: integrals restart at zero
    L1(rp::launch_zero(d_int, 2 * R, st), "zero integrals");
    if (!o.deterministic)
      L1(rp::launch_coherent_amps<T>(SYS, d_sample, nullptr, rows, seed, amps, nullptr, st),
         "amplitudes");
    L1(rp::launch_init_state<T>(SYS, amps, d_sample, nullptr, d_win, rows, o.deterministic, S0, S1,
                                nullptr, nullptr, st),
       "initial states");
    T* Sb[2] = {S0, S1};
    for (long long k = 0; k < max_macro; ++k) {
      T* P = Sb[k & 1];
      T* Q = Sb[(k + 1) & 1];
      T* phi[3] = {P, F1, F2};
      long long act = 0;
      for (int r = 0; r < rows; ++r) act += (k < h_win[r].y) ? 1 : 0;
      for (int n = 1; n < n_c; ++n) {
        const int mode = (n == 1) ? rp::MODE_FIRST : (n == n_c - 1 ? rp::MODE_LAST : rp::MODE_MID);
        L1(rp::launch_step<T>(SYS, &H, H.aniso, 0, d_fdev, d_field, d_win, (int)k, nullptr, rows,
                              phi[(n - 1) % 3],
                              n >= 2 ? phi[(n - 2) % 3] : nullptr,
                              mode == rp::MODE_LAST ? nullptr : phi[n % 3], Q, X, d_coef, n_c, n,
                              mode, 0, st),
           "step kernel");
        steps++;
      }
      row_terms += act * n_c;
      L1(rp::launch_gram_integrate<T>(SYS, X, d_W, d_field, d_win, (int)k, nullptr, rows, n_c,
                                      d_int, st),
         "gram-integral kernel");
    }
    L1(rp::launch_norm<T>(SYS, S0, S1, d_win, nullptr, rows, d_surv, st), "norm kernel");
    rp::RowsDev RD{d_field, d_win, d_sample, d_out, nullptr, d_int, d_surv};
    L1(rp::launch_finalize<T>(SYS, RD, rows, d_ps, st), "finalize kernel");
  }
  {
    std::vector<long long> offcnt(2 * (size_t)n_fields);
    for (int f = 0; f < n_fields; ++f) {
      offcnt[f] = (long long)f * Mr;
      offcnt[n_fields + f] = Mr;
    }
    sck(cudaMemcpyAsync(d_offcnt, offcnt.data(), offcnt.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    h2d += (long long)(offcnt.size() * sizeof(long long));
    L1(rp::launch_stats(d_ps, d_offcnt, d_offcnt + n_fields, n_fields, d_stats, st), "stats kernel");
  }
  sck(cudaMemcpyAsync(out, d_stats, (size_t)n_fields * 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  d2h += (long long)n_fields * 5 * sizeof(double);
  if (per_sample) {
    sck(cudaMemcpyAsync(per_sample, d_ps, (size_t)items * 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    d2h += (long long)items * 3 * sizeof(double);
  }
  sck(cudaStreamSynchronize(st), "kernel execution");
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->kernel_launches = launches;
    stats->step_launches = steps;
    stats->row_terms = row_terms;
    stats->propagations = items;
    stats->rows = (int)R;
    stats->n_cheb = n_c;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
  }
  return RP_OK;
}

}  // namespace

extern "C" rp_status rp_yields_static(rp_system* s, int n_fields, const double* fields, int M,
                                      uint64_t seed, double t_max, const rp_options* opt,
                                      double* out, double* per_sample, rp_stats* stats) {
  rp::set_last_error("");
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (!s) return sfail(RP_EINVAL, "system is NULL");
  if (n_fields < 0) return sfail(RP_EINVAL, "n_fields must be >= 0");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return sfail(RP_EINVAL, "bad precision");
  if (o.deterministic < 0 || o.deterministic > 3) return sfail(RP_EINVAL, "deterministic must be 0, 1, 2 or 3");
  if (o.deterministic > 1)
    return sfail(RP_ENOTIMPL, "basis-state sampling (deterministic = 2) and the J_z-sector trace "
                              "(deterministic = 3) are served by rp_yields");
  // this entry point runs the per-term kernels with the CUDA-core integral,
  // eagerly: other launch choices are refused rather than silently ignored
  if (o.kernel != 0 && o.kernel != 1) return sfail(RP_ENOTIMPL, "rp_yields_static runs kernel = 1 only (0 or 1 accepted)");
  if (o.gram != 0 && o.gram != 1) return sfail(RP_ENOTIMPL, "rp_yields_static runs gram = 1 only (0 or 1 accepted)");
  if (o.graph != 0) return sfail(RP_ENOTIMPL, "rp_yields_static does not replay CUDA graphs (graph must be 0)");
  if (o.max_rows < 0) return sfail(RP_EINVAL, "max_rows must be >= 0");
  if (!o.deterministic && M < 2) return sfail(RP_EINVAL, "M must be >= 2 (the standard error needs it)");
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return sfail(RP_EINVAL, "t_max must be positive and finite");
  if (o.sample_offset < 0) return sfail(RP_EINVAL, "sample_offset must be >= 0");
  if (n_fields > 0 && (!fields || !out)) return sfail(RP_EINVAL, "NULL fields or out");
  for (int f = 0; f < n_fields; ++f)
    if (!std::isfinite(fields[f])) return sfail(RP_EINVAL, "non-finite field");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_fields == 0) return RP_OK;
  unsigned char* scratch = nullptr;
  rp_status a = scratch_address(&scratch);
  if (a != RP_OK) return a;
  try {
    if (o.precision == RP_FP64)
      return run_static<double>(s->hs, n_fields, fields, M, seed, t_max, o, out, per_sample, stats, scratch);
    return run_static<float>(s->hs, n_fields, fields, M, seed, t_max, o, out, per_sample, stats, scratch);
  } catch (const StaticFail& e) {
    return sfail(e.st, e.msg);
  }
}
