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
#include <chrono>
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

int default_ncheb(int) { return 88; }  // fastest measured in both precisions (rp_tune)

}  // namespace

namespace rp {
// Kernel path rp_yields takes for kernel = 0 on one FP32 system (rp_tune's
// baseline), and whether the cluster path (kernel = 4) applies to it.
int default_kernel_fp32(const HostSystem& hs, bool* cluster_ok) {
  const HamDev<float> hf = make_ham<float>(hs);
  const bool ok = macro_cluster_plan(hf, nullptr);
  if (cluster_ok) *cluster_ok = ok;
  if (hs.Z <= small_max_configs<float>()) return persistent_default(hs.Z, 1) ? 5 : 2;
  return macro_cluster_default(hf) ? 4 : 1;
}

// kernel = 0 runs the persistent launch (kernel 5) for systems that fit one
// CTA with 128 <= Z <= 1024, and for batches of several such systems up to
// the size limit (measured faster than the on-chip macro-step launches).
bool persistent_default(long long Zslot, int n_systems) {
  return Zslot >= 128 && (Zslot <= 1024 || n_systems > 1);
}
}  // namespace rp

namespace {

bool bad_kernel_choice(const rp_options& o) {
  return o.kernel < 0 || o.kernel > 5 || o.graph < 0 || o.graph > 1 || o.gram < 0 || o.gram > 2;
}
double default_tol(int precision) { return precision == RP_FP64 ? 1e-15 : 1e-9; }

// One work item: a (field, sample) propagation over the whole horizon.
struct Item {
  int field;         // index into the engine's per-field tables
  long long sample;  // Philox sample index, or basis index when deterministic
  long long out;     // slot in the per-sample output array
  int n_macro;       // macro-steps of its field's plan
  int sys;           // index into the engine's systems
};

// Runs lists of work items on a pool of R rows: every row propagates one item
// through its macro-steps; when an item finishes, the row's survival and
// yields are written and the row takes the next item at the next macro-step
// (the schedule is known on the host from the per-field plans, so no
// device-to-host traffic is needed to refill).
template <typename T>
class YieldEngine {
 public:
  YieldEngine(const std::vector<const rp::HostSystem*>& systems, const rp_options& o, int n_c,
              cudaStream_t st, Arena& ar, const std::vector<uint32_t>* pairs = nullptr)
      : sys_(systems), o_(o), n_c_(n_c), st_(st), ar_(ar) {
    const int ns = (int)systems.size();
    std::vector<rp::HamDev<T>> ham(ns);
    std::vector<rp::LayoutDev> lay(ns);
    std::vector<double> kS(ns);
    Zslot_ = 1;
    ham1_ = make_ham<T>(*systems[0]);
    for (int i = 0; i < ns; ++i) {
      ham[i] = make_ham<T>(*systems[i]);
      lay[i] = make_layout(*systems[i]);
      kS[i] = systems[i]->k_S;
      Zslot_ = std::max<long long>(Zslot_, systems[i]->Z);
      aniso_ = aniso_ || systems[i]->aniso;
    }
    d_ham_ = ar_.get<rp::HamDev<T>>(ns);
    d_lay_ = ar_.get<rp::LayoutDev>(ns);
    d_kS_ = ar_.get<double>(ns);
    ck(cudaMemcpyAsync(d_ham_, ham.data(), ns * sizeof(ham[0]), cudaMemcpyHostToDevice, st_), "h2d systems");
    ck(cudaMemcpyAsync(d_lay_, lay.data(), ns * sizeof(lay[0]), cudaMemcpyHostToDevice, st_), "h2d systems");
    ck(cudaMemcpyAsync(d_kS_, kS.data(), ns * sizeof(double), cudaMemcpyHostToDevice, st_), "h2d systems");
    h2d += (long long)(ns * (sizeof(ham[0]) + sizeof(lay[0]) + sizeof(double)));
    if (pairs) {
      d_pair_ = ar_.get<uint32_t>(ns);
      ck(cudaMemcpyAsync(d_pair_, pairs->data(), ns * sizeof(uint32_t), cudaMemcpyHostToDevice, st_), "h2d pairs");
      h2d += (long long)(ns * sizeof(uint32_t));
    }
  }

  long long launches = 0, step_launches = 0, row_terms = 0, h2d = 0, d2h = 0;
  double step_bytes_all = 0.0;
  std::vector<cudaEvent_t> pev;
  std::vector<double> pev_bytes;
  std::vector<long long> pev_launches;

  ~YieldEngine() {
    for (auto e : pev) cudaEventDestroy(e);
    drop_graphs();
    if (cap_st_) cudaStreamDestroy(cap_st_);
    if (side_st_) {
      cudaStreamSynchronize(side_st_);
      cudaStreamDestroy(side_st_);
    }
    for (int i = 0; i < 2; ++i) {
      if (ev_step_[i]) cudaEventDestroy(ev_step_[i]);
      if (ev_int_[i]) cudaEventDestroy(ev_int_[i]);
    }
  }

  void set_fields(const std::vector<rp::FieldPlan>& plans) {
    const int nf = (int)plans.size();
    d_fdev_ = ar_.get<rp::FieldDev<T>>(nf);
    d_coef_ = ar_.get<T>((size_t)nf * n_c_ * 4);
    d_W_ = ar_.get<double>((size_t)nf * n_c_ * n_c_ * 2);
    std::vector<rp::FieldDev<T>> fdev(nf);
    // per field: c_n (re, im) in T, then the remainder c_n - fl(c_n) (FP32
    // only: the kernels add it, so the coefficients act with FP64 accuracy)
    std::vector<T> coef((size_t)nf * n_c_ * 4, T(0));
    std::vector<double> W((size_t)nf * n_c_ * n_c_ * 2);
    for (int f = 0; f < nf; ++f) {
      const rp::FieldPlan& P = plans[f];
      fdev[f].omega = (T)P.omega;
      fdev[f].s = (T)(1.0 / P.dE);
      fdev[f].sh_re = (T)(P.E_c / P.dE);
      fdev[f].sh_im = (T)0;
      for (int n = 0; n < n_c_; ++n) {
        const T re = (T)P.coef[n].real(), im = (T)P.coef[n].imag();
        T* cf = &coef[(size_t)f * n_c_ * 4];
        cf[2 * n] = re;
        cf[2 * n + 1] = im;
        if (sizeof(T) == 4) {
          cf[2 * n_c_ + 2 * n] = (T)(P.coef[n].real() - (double)re);
          cf[2 * n_c_ + 2 * n + 1] = (T)(P.coef[n].imag() - (double)im);
        }
      }
      for (size_t i = 0; i < (size_t)n_c_ * n_c_; ++i) {
        W[((size_t)f * n_c_ * n_c_ + i) * 2] = P.W[i].real();
        W[((size_t)f * n_c_ * n_c_ + i) * 2 + 1] = P.W[i].imag();
      }
    }
    ck(cudaMemcpyAsync(d_fdev_, fdev.data(), fdev.size() * sizeof(fdev[0]), cudaMemcpyHostToDevice, st_), "h2d fields");
    ck(cudaMemcpyAsync(d_coef_, coef.data(), coef.size() * sizeof(T), cudaMemcpyHostToDevice, st_), "h2d coef");
    ck(cudaMemcpyAsync(d_W_, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st_), "h2d W");
    h2d += (long long)(fdev.size() * sizeof(fdev[0]) + coef.size() * sizeof(T) + W.size() * sizeof(double));
  }

  static size_t row_bytes(long long Z, int n_c) {
    const size_t x_row = std::max<size_t>((size_t)n_c * Z * 2, rp::xblk_floats_per_row(Z, n_c));
    return (4 * (size_t)Z * 8 + x_row) * sizeof(T) + 256 + rp::kMaxNucDev * 20 * 8;
  }

  long long zslot() const { return Zslot_; }

  void alloc_rows(int R) {
    R_ = R;
    // one persistent launch over all items (kernel = 5) where every system
    // fits one CTA's shared memory; kernel = 5 elsewhere selects as 0.
    // kernel = 0 (without graph replay, which asks for macro-step launches)
    // takes it where it measured faster than one launch per macro-step:
    // 128 <= Z <= 1024, and batches of several systems
    const bool fits = Zslot_ <= rp::small_max_configs<T>() && o_.deterministic != 3 && !d_trace_;
    persist_ = fits && (o_.kernel == 5 || (o_.kernel == 0 && !o_.graph &&
                                           rp::persistent_default(Zslot_, (int)sys_.size())));
    d_err_ = ar_.get<int>(1);
    ck(cudaMemsetAsync(d_err_, 0, sizeof(int), st_), "cudaMemsetAsync");
    if (persist_) {
      pctas_ = rp::persistent_ctas<T>(Zslot_, n_c_, aniso_);
      if (pctas_ <= 0) throw CudaFail{RP_ECUDA, "persistent kernel: no device"};
      Xp_ = ar_.get<T>((size_t)pctas_ * n_c_ * Zslot_ * 2);
      d_counter_ = ar_.get<int>(1);
      S_ = rp::SysTab<T>{d_ham_, d_lay_, d_kS_, nullptr, Zslot_, o_.pair_id, d_pair_, d_err_,
                         sec_rank_, sec_scale_};
      return;
    }
    const int kq = o_.kernel == 5 ? 0 : o_.kernel;
    const size_t vec = (size_t)Zslot_ * 8;
    S0_ = ar_.get<T>((size_t)R * vec);
    S1_ = ar_.get<T>((size_t)R * vec);
    F1_ = ar_.get<T>((size_t)R * vec);
    F2_ = ar_.get<T>((size_t)R * vec);
    amps_ = ar_.get<double>((size_t)R * rp::kMaxNucDev * 10 * 2);
    row_sys_ = ar_.get<int>(R);
    small_ = (kq == 2 || (kq == 0 && Zslot_ <= rp::small_max_configs<T>())) &&
             Zslot_ <= rp::small_max_configs<T>();
    // a whole macro-step per launch on a thread-block cluster per row (FP32,
    // one isotropic system whose state fits the cluster's shared memory)
    cluster_ = false;
    if (sizeof(T) == 4 && !small_ && sys_.size() == 1 && (kq == 4 || kq == 0)) {
      const auto& hf = *reinterpret_cast<const rp::HamDev<float>*>(&ham1_);
      cluster_ = (kq == 4 ? rp::macro_cluster_plan(hf, nullptr)
                                 : rp::macro_cluster_default(hf)) &&
                 rp::macro_cluster_max_active(hf) > 0;
    }
    // tensor-core time integral: FP32 with the per-term kernels (each row's
    // integral covers its own system's Z; the step kernel keeps the padding of
    // the last 16-configuration chunk at zero)
    tc_gram_ = sizeof(T) == 4 && !small_ && o_.gram != 1 && rp::gram_tc_supported(n_c_);
    const size_t x_row = std::max<size_t>((size_t)n_c_ * Zslot_ * 2,
                                          rp::xblk_floats_per_row(Zslot_, n_c_));
    X_ = ar_.get<T>((size_t)R * x_row);
    // cluster macro-steps leave SMs idle (clusters fill whole GPC pairs of 8):
    // the time integral of macro-step k runs on a second stream, reading its own
    // copy of the singlet slices, while macro-step k + 1 propagates
    overlap_ = cluster_ && tc_gram_ && !o_.graph && !d_trace_;
    if (overlap_) {
      X2_ = ar_.get<T>((size_t)R * x_row);
      ck(cudaMemsetAsync(X2_, 0, (size_t)R * x_row * sizeof(T), st_), "cudaMemsetAsync");
      if (!side_st_) ck(cudaStreamCreateWithFlags(&side_st_, cudaStreamNonBlocking), "cudaStreamCreate");
      for (int i = 0; i < 2; ++i) {
        if (!ev_step_[i]) ck(cudaEventCreateWithFlags(&ev_step_[i], cudaEventDisableTiming), "cudaEventCreate");
        if (!ev_int_[i]) ck(cudaEventCreateWithFlags(&ev_int_[i], cudaEventDisableTiming), "cudaEventCreate");
      }
    }
    if (tc_gram_) {
      ck(cudaMemsetAsync(X_, 0, (size_t)R * x_row * sizeof(T), st_), "cudaMemsetAsync");
      int dev = 0;
      ck(cudaGetDevice(&dev), "cudaGetDevice");
      ck(cudaDeviceGetAttribute(&n_sm_, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    }
    S_ = rp::SysTab<T>{d_ham_, d_lay_, d_kS_, row_sys_, Zslot_, o_.pair_id, d_pair_, d_err_,
                       sec_rank_, sec_scale_};
    rows_.field = ar_.get<int>(R);
    rows_.win = ar_.get<int2>(R);
    rows_.sample = ar_.get<long long>(R);
    rows_.out = ar_.get<long long>(R);
    rows_.flag = ar_.get<int>(R);
    rows_.integral = ar_.get<double>(2 * (size_t)R);
    rows_.survival = rows_.integral + R;
  }

  // All items in one launch of k_persistent_small: CTAs take items from a
  // device counter, so nothing returns to the host until the last one ends.
  void run_persistent(const std::vector<Item>& items, double* d_ps) {
    const long long n = (long long)items.size();
    if (n == 0) return;
    if (n > 2000000000LL) throw CudaFail{RP_EINVAL, "too many propagations for one launch"};
    std::vector<rp::PItem> h((size_t)n);
    std::vector<double> cost((size_t)n);
    for (long long i = 0; i < n; ++i) {
      const Item& it = items[(size_t)i];
      h[(size_t)i] = rp::PItem{it.field, it.sys, it.n_macro, 0, it.sample, it.out};
      cost[(size_t)i] = (double)it.n_macro * (double)sys_[it.sys]->Z;
      row_terms += (long long)it.n_macro * n_c_;
      // HBM: the singlet slices out and back in per macro-step
      step_bytes_all += 2.0 * n_c_ * (double)sys_[it.sys]->Z * 2.0 * sizeof(T) * it.n_macro;
    }
    // longest items first (the CTAs take them in this order), so the launch
    // does not end on one long item started last
    std::vector<size_t> ord((size_t)n);
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
    std::vector<rp::PItem> hs((size_t)n);
    for (size_t i = 0; i < ord.size(); ++i) hs[i] = h[ord[i]];
    h.swap(hs);
    rp::PItem* d_items = ar_.get<rp::PItem>((size_t)n);
    ck(cudaMemcpyAsync(d_items, h.data(), h.size() * sizeof(rp::PItem), cudaMemcpyHostToDevice, st_),
       "h2d items");
    h2d += (long long)(h.size() * sizeof(rp::PItem));
    ck(cudaMemsetAsync(d_counter_, 0, sizeof(int), st_), "cudaMemsetAsync");
    if (o_.profile) {
      cudaEvent_t e0, e1;
      ck(cudaEventCreate(&e0), "cudaEventCreate");
      pev.push_back(e0);
      ck(cudaEventCreate(&e1), "cudaEventCreate");
      pev.push_back(e1);
      ck(cudaEventRecord(e0, st_), "cudaEventRecord");
    }
    launched(rp::launch_persistent_small<T>(S_, aniso_, d_fdev_, d_coef_, d_W_, d_items, (int)n,
                                            d_counter_, n_c_, o_.deterministic, seed_, Xp_, pctas_,
                                            d_ps, st_),
             "persistent kernel");
    step_launches += 1;
    if (o_.profile) {
      ck(cudaEventRecord(pev.back(), st_), "cudaEventRecord");
      pev_bytes.push_back(step_bytes_all);
      pev_launches.push_back(1);
    }
    ck(cudaStreamSynchronize(st_), "kernel execution");
  }

  void run(const std::vector<Item>& items, double* d_ps) {
    if (persist_) {
      run_persistent(items, d_ps);
      return;
    }
    const int R = R_;
    if (d_trace_ || o_.graph) overlap_ = false;  // eager, single-stream macro-steps
    const long long n_items = (long long)items.size();
    std::vector<int> h_field(R, 0), h_flag(R, 0), h_sys(R, 0);
    std::vector<int2> h_win(R, make_int2(0, 0));
    std::vector<long long> h_sample(R, 0), h_out(R, 0);
    long long next = 0;
    int live = 0;
    auto assign = [&](int r, int k) {
      const Item& it = items[next++];
      h_field[r] = it.field;
      h_win[r] = make_int2(k, k + it.n_macro);
      h_sample[r] = it.sample;
      h_out[r] = it.out;
      h_sys[r] = it.sys;
      h_flag[r] = 1;
    };
    auto upload_rows = [&]() {
      ck(cudaMemcpyAsync(rows_.field, h_field.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_), "h2d rows");
      ck(cudaMemcpyAsync(rows_.win, h_win.data(), R * sizeof(int2), cudaMemcpyHostToDevice, st_), "h2d rows");
      ck(cudaMemcpyAsync(rows_.sample, h_sample.data(), R * sizeof(long long), cudaMemcpyHostToDevice, st_), "h2d rows");
      ck(cudaMemcpyAsync(rows_.out, h_out.data(), R * sizeof(long long), cudaMemcpyHostToDevice, st_), "h2d rows");
      ck(cudaMemcpyAsync(rows_.flag, h_flag.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_), "h2d rows");
      ck(cudaMemcpyAsync(row_sys_, h_sys.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_), "h2d rows");
      h2d += (long long)R * (3 * sizeof(int) + sizeof(int2) + 2 * sizeof(long long));
    };
    auto init_flagged = [&]() {
      if (!o_.deterministic)
        launched(rp::launch_coherent_amps<T>(S_, rows_.sample, rows_.flag, R, seed_, amps_, nullptr,
                                             st_), "coherent amplitudes");
      launched(rp::launch_init_state<T>(S_, amps_, rows_.sample, rows_.flag, rows_.win, R,
                                        o_.deterministic, S0_, S1_, rows_.integral,
                                        rows_.survival, st_), "initial states");
    };
    for (int r = 0; r < R && next < n_items; ++r) {
      assign(r, 0);
      ++live;
    }
    upload_rows();
    init_flagged();
    if (o_.graph) {
      if (!d_macro_) d_macro_ = ar_.get<int>(1);
      ck(cudaMemsetAsync(d_macro_, 0, sizeof(int), st_), "cudaMemsetAsync");
      drop_graphs();
    }
    for (int k = 0; live > 0; ++k) {
      long long act = 0;
      double act_z = 0.0;  // configurations of the active rows
      for (int r = 0; r < R; ++r)
        if (h_win[r].x <= k && k < h_win[r].y) {
          ++act;
          act_z += (double)sys_[h_sys[r]]->Z;
        }
      const double vbytes = 8.0 * sizeof(T) * act_z;  // one state vector of every active row
      if (o_.profile) {
        cudaEvent_t a, b;
        ck(cudaEventCreate(&a), "cudaEventCreate");
        pev.push_back(a);
        ck(cudaEventCreate(&b), "cudaEventCreate");
        pev.push_back(b);
        ck(cudaEventRecord(a, st_), "cudaEventRecord");
      }
      double bytes = 0.0;
      if (small_ || cluster_) {
        // the whole macro-step on chip: HBM traffic is psi in, psi out and the singlet slices
        bytes = (2.0 + 0.25 * n_c_) * vbytes;
      } else {
        for (int n = 1; n < n_c_; ++n) bytes += rp::term_vector_passes(n, n_c_) * vbytes;
      }
      // profile events bracket the step kernels (eager) or the whole graph replay
      cudaEvent_t ev_end = o_.profile ? pev.back() : nullptr;
      int n_step = 0;
      if (!o_.graph || d_trace_) {
        n_step = issue(k, st_, nullptr, ev_end);
        launches += n_step + 1;
      } else if (k < 2) {
        // the first macro-step of each parity runs eagerly (kernel attributes get set)
        n_step = issue(k, st_, d_macro_, ev_end);
        launches += n_step + 2;
      } else {
        const int p = k & 1;
        if (!gexec_[p]) capture(k, p);
        ck(cudaGraphLaunch(gexec_[p], st_), "cudaGraphLaunch");
        if (ev_end) ck(cudaEventRecord(ev_end, st_), "cudaEventRecord");
        n_step = gsteps_[p];
        launches += n_step + 2;
        graph_launches++;
      }
      step_launches += n_step;
      if (o_.profile) {
        pev_bytes.push_back(bytes);
        pev_launches.push_back(n_step);
      }
      step_bytes_all += bytes;
      row_terms += act * (long long)n_c_;
      if (d_trace_) {
        T* Sb2[2] = {S0_, S1_};
        launched(rp::launch_trace<T>(S_, Sb2[(k + 1) & 1], rows_.win, k, R_, trace_op_, d_trace_, st_),
                 "trace kernel");
      }
      // rows whose window ends after this macro-step: finish and refill
      bool any = false;
      for (int r = 0; r < R; ++r) {
        h_flag[r] = (h_win[r].y == k + 1 && h_win[r].x <= k) ? 1 : 0;
        any = any || h_flag[r];
      }
      if (!any) continue;
      // the finishing rows' integrals (and every row's metadata the side
      // stream still reads) are complete once macro-step k is integrated
      if (overlap_) ck(cudaStreamWaitEvent(st_, ev_int_[k & 1], 0), "cudaStreamWaitEvent");
      ck(cudaMemcpyAsync(rows_.flag, h_flag.data(), R * sizeof(int), cudaMemcpyHostToDevice, st_), "h2d flags");
      h2d += (long long)R * sizeof(int);
      launched(rp::launch_norm<T>(S_, S0_, S1_, rows_.win, rows_.flag, R, rows_.survival, st_), "norm kernel");
      launched(rp::launch_finalize<T>(S_, rows_, R, d_ps, st_), "finalize kernel");
      bool refill = false;
      for (int r = 0; r < R; ++r) {
        if (!h_flag[r]) continue;
        if (next < n_items) {
          assign(r, k + 1);
          refill = true;
        } else {
          h_flag[r] = 0;
          --live;
        }
      }
      if (refill) {
        upload_rows();
        init_flagged();
      }
    }
    drop_graphs();
    if (overlap_) {
      // everything on the side stream before the caller's stream goes on
      ck(cudaEventRecord(ev_int_[0], side_st_), "cudaEventRecord");
      ck(cudaStreamWaitEvent(st_, ev_int_[0], 0), "cudaStreamWaitEvent");
    }
    // kernels with bounded waits report a wait that gave up in the error word
    int h_err = 0;
    ck(cudaMemcpyAsync(&h_err, d_err_, sizeof(int), cudaMemcpyDeviceToHost, st_), "d2h error word");
    d2h += (long long)sizeof(int);
    ck(cudaStreamSynchronize(st_), "kernel execution");
    if (h_err) throw CudaFail{RP_ETIMEOUT, "a bounded device wait gave up (bulk tile copies)"};
  }

  void set_seed(uint64_t seed) { seed_ = seed; }

  // J_z-sector tables of deterministic = 3 (device arrays; before alloc_rows).
  void set_sectors(const int* rank, const double* scale) {
    sec_rank_ = rank;
    sec_scale_ = scale;
  }

  // Kernel path taken (rp_stats.kernel_path): 5 persistent, 4 cluster, 2 one
  // CTA per row, 3 staged per-term, 1 per-term.
  int kernel_path() const {
    return persist_ ? 5 : cluster_ ? 4 : (small_ ? 2 : (o_.kernel == 3 ? 3 : 1));
  }
  // Rows propagated at once: CTAs of the persistent launch, else allocated rows.
  int rows_used() const { return persist_ ? pctas_ : R_; }

  // Time-resolved sums (launch_trace) after every macro-step, 4 doubles per
  // time point, with an optional electron operator; eager launches.
  void set_trace(double* trace, const rp::ElecOp& op) {
    d_trace_ = trace;
    trace_op_ = op;
  }

  long long graph_launches = 0;

 private:
  void launched(cudaError_t e, const char* what) {
    ck(e, what);
    launches++;
  }

  // Launches the macro-step k on stream s: the Chebyshev terms (one kernel per
  // term, or the whole macro-step in shared memory), the time integral and,
  // with a device counter mdev, the counter increment.  Returns the number of
  // step-kernel launches.
  int issue(int k, cudaStream_t s, int* mdev, cudaEvent_t ev_steps = nullptr) {
    T* Sb[2] = {S0_, S1_};
    T* P = Sb[k & 1];
    T* Q = Sb[(k + 1) & 1];
    T* phi[3] = {P, F1_, F2_};
    const rp::HamDev<T>* one = sys_.size() == 1 ? &ham1_ : nullptr;
    int n_step = 0;
    if (small_) {
      ck(rp::launch_macro_small<T>(S_, one, aniso_, d_fdev_, rows_.field, rows_.win, k, mdev, R_,
                                   P, Q, X_, d_coef_, n_c_, s),
         "macro-step kernel");
      n_step = 1;
    }
    T* Xk = (overlap_ && (k & 1)) ? X2_ : X_;
    if (cluster_) {
      // the slices of macro-step k - 2 (same buffer) must have been integrated
      if (overlap_ && k >= 2) ck(cudaStreamWaitEvent(s, ev_int_[k & 1], 0), "cudaStreamWaitEvent");
      ck(rp::launch_macro_cluster(*reinterpret_cast<const rp::HamDev<float>*>(&ham1_),
                                  reinterpret_cast<const rp::FieldDev<float>*>(d_fdev_),
                                  rows_.field, rows_.win, k, mdev, R_,
                                  reinterpret_cast<const float*>(P), reinterpret_cast<float*>(Q),
                                  reinterpret_cast<float*>(Xk),
                                  reinterpret_cast<const float*>(d_coef_), n_c_, Zslot_,
                                  tc_gram_ ? 1 : 0, s),
         "cluster macro-step kernel");
      n_step = 1;
    }
    for (int n = 1; n < n_c_ && !small_ && !cluster_; ++n) {
      const int mode = (n == 1) ? rp::MODE_FIRST : (n == n_c_ - 1 ? rp::MODE_LAST : rp::MODE_MID);
      ck(rp::launch_step<T>(S_, one, aniso_, o_.kernel == 3, d_fdev_, rows_.field, rows_.win, k, mdev, R_,
                            phi[(n - 1) % 3], n >= 2 ? phi[(n - 2) % 3] : nullptr,
                            mode == rp::MODE_LAST ? nullptr : phi[n % 3], Q, X_, d_coef_, n_c_, n,
                            mode, tc_gram_ ? 1 : 0, s),
         "step kernel");
      ++n_step;
    }
    if (ev_steps) ck(cudaEventRecord(ev_steps, s), "cudaEventRecord");
    if (overlap_) {
      ck(cudaEventRecord(ev_step_[k & 1], s), "cudaEventRecord");
      ck(cudaStreamWaitEvent(side_st_, ev_step_[k & 1], 0), "cudaStreamWaitEvent");
      ck(rp::launch_gram_tc(reinterpret_cast<const float*>(Xk), d_W_, rows_.field, rows_.win, k,
                            mdev, R_, n_c_, Zslot_,
                            reinterpret_cast<const rp::HamDev<float>*>(d_ham_),
                            sys_.size() == 1 ? nullptr : row_sys_, n_sm_, rows_.integral, d_err_,
                            side_st_),
         "tensor-core time-integral kernel");
      ck(cudaEventRecord(ev_int_[k & 1], side_st_), "cudaEventRecord");
    } else if (tc_gram_)
      ck(rp::launch_gram_tc(reinterpret_cast<const float*>(X_), d_W_, rows_.field, rows_.win, k,
                            mdev, R_, n_c_, Zslot_,
                            reinterpret_cast<const rp::HamDev<float>*>(d_ham_),
                            sys_.size() == 1 ? nullptr : row_sys_, n_sm_, rows_.integral, d_err_,
                            s),
         "tensor-core time-integral kernel");
    else
      ck(rp::launch_gram_integrate<T>(S_, X_, d_W_, rows_.field, rows_.win, k, mdev, R_, n_c_,
                                      rows_.integral, s),
         "gram-integral kernel");
    if (mdev) ck(rp::launch_tick(mdev, s), "tick kernel");
    return n_step;
  }

  // Records the launches of a macro-step of parity p (k % 2 == p) into a graph.
  void capture(int k, int p) {
    if (!cap_st_) ck(cudaStreamCreateWithFlags(&cap_st_, cudaStreamNonBlocking), "cudaStreamCreate");
    ck(cudaStreamBeginCapture(cap_st_, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaGraph_t g = nullptr;
    try {
      gsteps_[p] = issue(k, cap_st_, d_macro_);
    } catch (...) {
      cudaStreamEndCapture(cap_st_, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    ck(cudaStreamEndCapture(cap_st_, &g), "cudaStreamEndCapture");
    cudaError_t e = cudaGraphInstantiate(&gexec_[p], g, 0);
    cudaGraphDestroy(g);
    ck(e, "cudaGraphInstantiate");
  }

  void drop_graphs() {
    for (int p = 0; p < 2; ++p)
      if (gexec_[p]) {
        cudaGraphExecDestroy(gexec_[p]);
        gexec_[p] = nullptr;
      }
  }

  int* d_err_ = nullptr;
  double* d_trace_ = nullptr;
  cudaGraphExec_t gexec_[2] = {nullptr, nullptr};
  int gsteps_[2] = {0, 0};
  cudaStream_t cap_st_ = nullptr;
  int* d_macro_ = nullptr;
  std::vector<const rp::HostSystem*> sys_;
  const rp_options& o_;
  int n_c_;
  cudaStream_t st_;
  Arena& ar_;
  long long Zslot_ = 1;
  int aniso_ = 0;
  rp::HamDev<T>* d_ham_ = nullptr;
  rp::LayoutDev* d_lay_ = nullptr;
  double* d_kS_ = nullptr;
  int* row_sys_ = nullptr;
  uint32_t* d_pair_ = nullptr;
  rp::HamDev<T> ham1_{};
  bool small_ = false;
  bool cluster_ = false;
  bool overlap_ = false;
  bool persist_ = false;
  int pctas_ = 0;
  T* Xp_ = nullptr;
  int* d_counter_ = nullptr;
  T* X2_ = nullptr;
  cudaStream_t side_st_ = nullptr;
  cudaEvent_t ev_step_[2] = {nullptr, nullptr}, ev_int_[2] = {nullptr, nullptr};
  const int* sec_rank_ = nullptr;
  const double* sec_scale_ = nullptr;
  rp::ElecOp trace_op_{};
  bool tc_gram_ = false;
  int n_sm_ = 0;
  rp::SysTab<T> S_{};
  uint64_t seed_ = 0;
  int R_ = 0;
  rp::FieldDev<T>* d_fdev_ = nullptr;
  T* d_coef_ = nullptr;
  double* d_W_ = nullptr;
  T *S0_ = nullptr, *S1_ = nullptr, *F1_ = nullptr, *F2_ = nullptr, *X_ = nullptr;
  double* amps_ = nullptr;
  rp::RowsDev rows_{};
};

// Rows to allocate: the caller's cap, else 45 % of free device memory.
template <typename T>
int choose_rows(const rp::HostSystem& hs, const rp_options& o, int n_c, long long items) {
  long long cap = o.max_rows > 0 ? o.max_rows : 0;
  if (cap == 0) {
    size_t fr = 0, tot = 0;
    ck(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    cap = std::max<long long>(1, (long long)(0.45 * (double)fr / (double)YieldEngine<T>::row_bytes(hs.Z, n_c)));
  }
  cap = std::min<long long>(cap, 65535);
  return (int)std::max<long long>(1, std::min<long long>(items, cap));
}

// Sample identity of item s: 0 coherent-state sample index sample_offset + s;
// 1 basis index s (the trace, Eq. 14); 2 a basis index drawn for sample
// sample_offset + s (rp::basis_draw).
struct SampleMode {
  int mode = 0;
  uint64_t seed = 0;
  uint32_t pair = 0;
  long long Z = 1;
};

std::vector<Item> make_items(const std::vector<rp::FieldPlan>& plans, const std::vector<long long>& first,
                             const std::vector<long long>& count, const std::vector<long long>& out0,
                             long long sample_offset, SampleMode sm,
                             const std::vector<int>* sys_of_field = nullptr) {
  // most expensive fields first, so that rows finish in waves
  std::vector<int> forder(plans.size());
  for (size_t f = 0; f < plans.size(); ++f) forder[f] = (int)f;
  std::stable_sort(forder.begin(), forder.end(),
                   [&](int a, int b) { return plans[a].n_macro > plans[b].n_macro; });
  std::vector<Item> items;
  for (int f : forder)
    for (long long s = first[f]; s < first[f] + count[f]; ++s)
      items.push_back(Item{f,
                           (sm.mode == 1 || sm.mode == 3) ? s
                           : sm.mode == 2 ? rp::basis_draw(sm.seed, sm.pair, sample_offset + s, sm.Z)
                                          : sample_offset + s,
                           out0[f] + (s - first[f]), (int)plans[f].n_macro,
                           sys_of_field ? (*sys_of_field)[f] : 0});
  return items;
}

rp_status plan_all(const rp::HostSystem& hs, int n_fields, const double* fields, double t_max,
                   int n_c, double tol, std::vector<rp::FieldPlan>& plans) {
  plans.resize(n_fields);
  for (int f = 0; f < n_fields; ++f) {
    std::string e = rp::plan_field(hs, fields[f], t_max, n_c, tol, true, &plans[f]);
    if (!e.empty()) return fail(RP_ENOTCONV, "field " + std::to_string(f) + ": " + e);
    if (plans[f].n_macro > 2000000000LL) return fail(RP_ENOTCONV, "too many macro-steps");
  }
  return RP_OK;
}

template <typename T>
void fill_stats(rp_stats* stats, const YieldEngine<T>& eng, long long items, int R, int n_c,
                cudaEvent_t ev0, cudaEvent_t ev1, bool profile, long long d2h) {
  if (!stats) return;
  std::memset(stats, 0, sizeof(*stats));
  stats->kernel_launches = eng.launches;
  stats->step_launches = eng.step_launches;
  stats->graph_launches = eng.graph_launches;
  stats->row_terms = eng.row_terms;
  stats->propagations = items;
  stats->rows = eng.kernel_path() == 5 ? eng.rows_used() : R;
  stats->n_cheb = n_c;
  stats->kernel_path = eng.kernel_path();
  float ms = 0.f;
  ck(cudaEventElapsedTime(&ms, ev0, ev1), "cudaEventElapsedTime");
  stats->device_ms = ms;
  double pms = 0.0, pb = 0.0;
  long long pl = 0;
  for (size_t i = 0; i + 1 < eng.pev.size(); i += 2) {
    float t = 0.f;
    ck(cudaEventElapsedTime(&t, eng.pev[i], eng.pev[i + 1]), "cudaEventElapsedTime");
    pms += t;
    pb += eng.pev_bytes[i / 2];
    pl += eng.pev_launches[i / 2];
  }
  stats->step_ms = pms;
  stats->step_bytes = profile ? pb : eng.step_bytes_all;
  stats->step_launches_timed = pl;
  stats->h2d_bytes = eng.h2d;
  stats->d2h_bytes = d2h + eng.d2h;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    ck(cudaEventCreate(&a), "cudaEventCreate");
    ck(cudaEventCreate(&b), "cudaEventCreate");
  }
  ~EventPair() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

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
  // J_z-sector trace: propagation i carries the i-th basis state of every
  // nuclear-M class, normalised; it counts n_i / Z in the trace (Eq. 14)
  std::vector<int> sec_rank, sec_n;
  const long long n_sec = o.deterministic == 3 ? rp::sector_table(hs, &sec_rank, &sec_n) : 0;
  const long long Mr = o.deterministic == 1 ? hs.Z : (o.deterministic == 3 ? n_sec : (long long)M);
  std::vector<rp::FieldPlan> plans;
  rp_status ps = plan_all(hs, n_fields, fields, t_max, n_c, tol, plans);
  if (ps != RP_OK) return ps;
  std::vector<long long> first(n_fields, 0), count(n_fields, Mr), out0(n_fields);
  for (int f = 0; f < n_fields; ++f) out0[f] = (long long)f * Mr;
  const std::vector<Item> items = make_items(plans, first, count, out0, o.sample_offset,
                                             SampleMode{o.deterministic, seed, o.pair_id, hs.Z});
  const long long n_items = (long long)items.size();
  const int R = choose_rows<T>(hs, o, n_c, n_items);

  EventPair ev;
  long long d2h = 0;
  {
    Arena ar(st);
    YieldEngine<T> eng({&hs}, o, n_c, st, ar);
    eng.set_seed(seed);
    ck(cudaEventRecord(ev.a, st), "cudaEventRecord");
    eng.set_fields(plans);
    double* d_w = nullptr;
    if (o.deterministic == 3) {
      int* d_rank = ar.get<int>(sec_rank.size());
      double* d_scale = ar.get<double>((size_t)n_sec);
      d_w = ar.get<double>((size_t)n_sec);
      std::vector<double> scale((size_t)n_sec), w((size_t)n_sec);
      for (long long i = 0; i < n_sec; ++i) {
        scale[(size_t)i] = 1.0 / std::sqrt((double)sec_n[(size_t)i]);
        w[(size_t)i] = (double)sec_n[(size_t)i] / (double)hs.Z;
      }
      ck(cudaMemcpyAsync(d_rank, sec_rank.data(), sec_rank.size() * sizeof(int), cudaMemcpyHostToDevice, st), "h2d sectors");
      ck(cudaMemcpyAsync(d_scale, scale.data(), scale.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d sectors");
      ck(cudaMemcpyAsync(d_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d sectors");
      eng.h2d += (long long)(sec_rank.size() * sizeof(int) + 2 * scale.size() * sizeof(double));
      eng.set_sectors(d_rank, d_scale);
    }
    eng.alloc_rows(R);
    double* d_ps = ar.get<double>((size_t)n_items * 3);
    double* d_stats = ar.get<double>((size_t)n_fields * 5);
    long long* d_off = ar.get<long long>(2 * (size_t)n_fields);
    eng.run(items, d_ps);
    std::vector<long long> offcnt(2 * (size_t)n_fields);
    for (int f = 0; f < n_fields; ++f) {
      offcnt[f] = out0[f];
      offcnt[n_fields + f] = Mr;
    }
    ck(cudaMemcpyAsync(d_off, offcnt.data(), offcnt.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    eng.h2d += (long long)(offcnt.size() * sizeof(long long));
    if (o.deterministic == 3)
      ck(rp::launch_stats_weighted(d_ps, d_off, d_off + n_fields, d_w, n_fields, d_stats, st),
         "weighted stats kernel");
    else
      ck(rp::launch_stats(d_ps, d_off, d_off + n_fields, n_fields, d_stats, st), "stats kernel");
    eng.launches++;
    ck(cudaMemcpyAsync(out, d_stats, (size_t)n_fields * 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h stats");
    d2h += (long long)n_fields * 5 * sizeof(double);
    if (per_sample) {
      ck(cudaMemcpyAsync(per_sample, d_ps, (size_t)n_items * 3 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h per-sample");
      d2h += (long long)n_items * 3 * sizeof(double);
    }
    ck(cudaEventRecord(ev.b, st), "cudaEventRecord");
    ck(cudaStreamSynchronize(st), "kernel execution");
    fill_stats(stats, eng, n_items, R, n_c, ev.a, ev.b, o.profile != 0, d2h);
  }
  ck(cudaStreamSynchronize(st), "free");
  return RP_OK;
}

// Time-resolved P_S(t), P_T(t) and survival (Eq. 18 with A = P_S, P_T, 1)
// at the macro-step boundaries t_i = i h of one field, averaged over the
// samples (or the Z basis states when deterministic).
template <typename T>
rp_status run_time_trace(rp_system* sys, double B, int M, uint64_t seed, double t_max,
                         const rp_options& o, int n_times, double* t, double* out,
                         const double* A_e = nullptr, double* obs = nullptr) {
  const rp::HostSystem& hs = sys->hs;
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  const double tol = o.tol > 0 ? o.tol : default_tol(o.precision);
  const long long Mr = o.deterministic == 1 ? hs.Z : (long long)M;
  std::vector<rp::FieldPlan> plans;
  rp_status ps = plan_all(hs, 1, &B, t_max, n_c, tol, plans);
  if (ps != RP_OK) return ps;
  std::vector<long long> first(1, 0), count(1, Mr), out0(1, 0);
  const std::vector<Item> items = make_items(plans, first, count, out0, o.sample_offset,
                                             SampleMode{o.deterministic, seed, o.pair_id, hs.Z});
  const int R = choose_rows<T>(hs, o, n_c, (long long)items.size());
  std::vector<double> h_tr(4 * (size_t)n_times, 0.0);
  rp::ElecOp op{};
  if (A_e) {
    for (int q = 0; q < 16; ++q) {
      op.re[q] = A_e[2 * q];
      op.im[q] = A_e[2 * q + 1];
    }
    op.on = 1;
  }
  {
    Arena ar(st);
    YieldEngine<T> eng({&hs}, o, n_c, st, ar);
    eng.set_seed(seed);
    eng.set_fields(plans);
    double* d_tr = ar.get<double>(4 * (size_t)n_times);
    ck(cudaMemsetAsync(d_tr, 0, 4 * (size_t)n_times * sizeof(double), st), "cudaMemsetAsync");
    eng.set_trace(d_tr, op);
    eng.alloc_rows(R);
    double* d_ps = ar.get<double>(items.size() * 3);
    eng.run(items, d_ps);
    ck(cudaMemcpyAsync(h_tr.data(), d_tr, h_tr.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
       "d2h trace");
    ck(cudaStreamSynchronize(st), "kernel execution");
  }
  ck(cudaStreamSynchronize(st), "free");
  const double h = plans[0].h;
  for (int i = 0; i < n_times; ++i) {
    t[i] = i * h;
    // psi(0) = |S> x (normalised nuclear state): P_S = survival = 1, P_T = 0
    const double p_s = i == 0 ? 1.0 : h_tr[4 * (size_t)i] / (double)Mr;
    const double surv = i == 0 ? 1.0 : h_tr[4 * (size_t)i + 1] / (double)Mr;
    if (out) {
      out[3 * (size_t)i] = p_s;
      out[3 * (size_t)i + 1] = surv - p_s;  // P_T = 1 - P_S on the electrons
      out[3 * (size_t)i + 2] = surv;
    }
    if (obs) {
      if (i == 0) {
        // <S| A |S> for the normalised initial states
        const double s = 0.70710678118654752440;
        const double v[4] = {0.0, s, -s, 0.0};
        double re = 0.0, im = 0.0;
        for (int e = 0; e < 4; ++e)
          for (int f = 0; f < 4; ++f) {
            re += v[e] * A_e[2 * (4 * e + f)] * v[f];
            im += v[e] * A_e[2 * (4 * e + f) + 1] * v[f];
          }
        obs[0] = re;
        obs[1] = im;
      } else {
        obs[2 * (size_t)i] = h_tr[4 * (size_t)i + 2] / (double)Mr;
        obs[2 * (size_t)i + 1] = h_tr[4 * (size_t)i + 3] / (double)Mr;
      }
    }
  }
  return RP_OK;
}

// Rounds of samples per field until each field's standard error (Eq. 23)
// reaches se_target: M_min samples everywhere first, then per field the
// samples its measured spread asks for, (sigma_f / se_target)^2 with a 15 %
// margin, capped at M_max.  Sample s is the same direction set at every field.
template <typename T>
rp_status run_converged(rp_system* sys, int n_fields, const double* fields, double se_target,
                        int M_min, int M_max, uint64_t seed, double t_max, const rp_options& o,
                        double* out, int* M_used, rp_stats* stats) {
  const rp::HostSystem& hs = sys->hs;
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  const double tol = o.tol > 0 ? o.tol : default_tol(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  std::vector<rp::FieldPlan> plans;
  rp_status ps = plan_all(hs, n_fields, fields, t_max, n_c, tol, plans);
  if (ps != RP_OK) return ps;
  std::vector<std::vector<double>> samp(n_fields);  // phi_S, phi_T, survival triples
  std::vector<long long> have(n_fields, 0), want(n_fields, M_min);
  EventPair ev;
  long long d2h = 0, total_items = 0;
  int R = 0;
  {
    Arena ar(st);
    YieldEngine<T> eng({&hs}, o, n_c, st, ar);
    eng.set_seed(seed);
    ck(cudaEventRecord(ev.a, st), "cudaEventRecord");
    eng.set_fields(plans);
    R = choose_rows<T>(hs, o, n_c, std::max<long long>((long long)n_fields * M_min, 256));
    eng.alloc_rows(R);
    for (int round = 0; round < 8; ++round) {
      std::vector<long long> first(n_fields), count(n_fields), out0(n_fields);
      long long n = 0;
      for (int f = 0; f < n_fields; ++f) {
        first[f] = have[f];
        count[f] = std::max<long long>(0, want[f] - have[f]);
        out0[f] = n;
        n += count[f];
      }
      if (n == 0) break;
      const std::vector<Item> items = make_items(plans, first, count, out0, o.sample_offset, SampleMode{});
      double* d_ps = ar.get<double>((size_t)n * 3);
      eng.run(items, d_ps);
      std::vector<double> h((size_t)n * 3);
      ck(cudaMemcpyAsync(h.data(), d_ps, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h round");
      ck(cudaStreamSynchronize(st), "round");
      d2h += (long long)h.size() * sizeof(double);
      total_items += n;
      for (int f = 0; f < n_fields; ++f) {
        samp[f].insert(samp[f].end(), h.begin() + out0[f] * 3, h.begin() + (out0[f] + count[f]) * 3);
        have[f] += count[f];
      }
      // next targets from the spread measured so far
      bool more = false;
      for (int f = 0; f < n_fields; ++f) {
        const long long m = have[f];
        double mean = 0.0, var = 0.0;
        for (long long i = 0; i < m; ++i) mean += samp[f][3 * i];
        mean /= (double)m;
        for (long long i = 0; i < m; ++i) var += (samp[f][3 * i] - mean) * (samp[f][3 * i] - mean);
        var /= (double)std::max<long long>(m - 1, 1);
        const double se = std::sqrt(var / (double)m);
        if (se <= se_target || m >= M_max) {
          want[f] = m;
          continue;
        }
        const long long need = (long long)std::ceil(1.15 * var / (se_target * se_target)) + 1;
        // at most 4x per round: the spread of few samples is itself uncertain
        want[f] = std::min<long long>({M_max, std::max<long long>(need, m + 1), 4 * m});
        more = true;
      }
      if (!more) break;
    }
    // final per-field statistics on the device over all rounds' samples
    long long tot = 0;
    std::vector<long long> offcnt(2 * (size_t)n_fields);
    for (int f = 0; f < n_fields; ++f) {
      offcnt[f] = tot;
      offcnt[n_fields + f] = have[f];
      tot += have[f];
    }
    std::vector<double> all;
    all.reserve((size_t)tot * 3);
    for (int f = 0; f < n_fields; ++f) all.insert(all.end(), samp[f].begin(), samp[f].end());
    double* d_all = ar.get<double>((size_t)std::max<long long>(tot, 1) * 3);
    long long* d_off = ar.get<long long>(2 * (size_t)n_fields);
    double* d_stats = ar.get<double>((size_t)n_fields * 5);
    ck(cudaMemcpyAsync(d_all, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
    ck(cudaMemcpyAsync(d_off, offcnt.data(), offcnt.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    eng.h2d += (long long)(all.size() * sizeof(double) + offcnt.size() * sizeof(long long));
    ck(rp::launch_stats(d_all, d_off, d_off + n_fields, n_fields, d_stats, st), "stats kernel");
    eng.launches++;
    ck(cudaMemcpyAsync(out, d_stats, (size_t)n_fields * 5 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h stats");
    d2h += (long long)n_fields * 5 * sizeof(double);
    ck(cudaEventRecord(ev.b, st), "cudaEventRecord");
    ck(cudaStreamSynchronize(st), "kernel execution");
    if (M_used)
      for (int f = 0; f < n_fields; ++f) M_used[f] = (int)have[f];
    fill_stats(stats, eng, total_items, R, n_c, ev.a, ev.b, o.profile != 0, d2h);
  }
  ck(cudaStreamSynchronize(st), "free");
  return RP_OK;
}

// Converged curve with the learned control variate (see rp_yields_cv in rp.h).
template <typename T>
rp_status run_converged_cv(rp_system* sys, int n_fields, const double* fields, double se_target,
                           int M_min, int M_max, uint64_t seed, double t_max, const rp_options& o,
                           const rp_cv_plan& cp, double* out, int* M_plain, int* M_cv,
                           rp_stats* stats) {
  const rp::HostSystem& hs = sys->hs;
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  const double tol = o.tol > 0 ? o.tol : default_tol(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  std::vector<rp::FieldPlan> plans;
  rp_status ps = plan_all(hs, n_fields, fields, t_max, n_c, tol, plans);
  if (ps != RP_OK) return ps;
  // control-variate samples live far above every plain sample index
  const long long kCvBase = 1LL << 40;
  const double se2 = se_target * se_target;
  std::vector<std::vector<double>> pl(n_fields), cvs(n_fields), cvg(n_fields);
  std::vector<long long> have(n_fields, 0), want(n_fields, M_min), have_cv(n_fields, 0);
  std::vector<char> is_cv(n_fields, 0);
  EventPair ev;
  long long d2h = 0, total_items = 0;
  int R = 0;
  rp_cv* cv = nullptr;
  struct CvGuard {
    rp_cv** p;
    ~CvGuard() {
      if (*p) rp_cv_destroy(*p);
    }
  } cvguard{&cv};
  auto plain_stats = [&](int f, double* mean, double* var) {
    const long long m = have[f];
    double a = 0.0, v = 0.0;
    for (long long i = 0; i < m; ++i) a += pl[f][3 * i];
    a /= (double)m;
    for (long long i = 0; i < m; ++i) v += (pl[f][3 * i] - a) * (pl[f][3 * i] - a);
    *mean = a;
    *var = v / (double)std::max<long long>(m - 1, 1);
  };
  {
    Arena ar(st);
    YieldEngine<T> eng({&hs}, o, n_c, st, ar);
    eng.set_seed(seed);
    ck(cudaEventRecord(ev.a, st), "cudaEventRecord");
    eng.set_fields(plans);
    R = choose_rows<T>(hs, o, n_c, std::max<long long>((long long)n_fields * M_min, 256));
    eng.alloc_rows(R);
    // run counts[f] new samples of field f starting at first[f]; per-sample results appended
    auto run_round = [&](const std::vector<long long>& first, const std::vector<long long>& count,
                         std::vector<std::vector<double>>& dst) {
      std::vector<long long> out0(n_fields);
      long long n = 0;
      for (int f = 0; f < n_fields; ++f) {
        out0[f] = n;
        n += count[f];
      }
      if (n == 0) return;
      const std::vector<Item> items = make_items(plans, first, count, out0, 0, SampleMode{});
      double* d_ps = ar.get<double>((size_t)n * 3);
      eng.run(items, d_ps);
      std::vector<double> h((size_t)n * 3);
      ck(cudaMemcpyAsync(h.data(), d_ps, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h round");
      ck(cudaStreamSynchronize(st), "round");
      d2h += (long long)h.size() * sizeof(double);
      total_items += n;
      for (int f = 0; f < n_fields; ++f)
        dst[f].insert(dst[f].end(), h.begin() + out0[f] * 3, h.begin() + (out0[f] + count[f]) * 3);
    };
    // 1. plain pilot, then plain rounds for fields below the control-variate threshold and
    //    plain training samples for the others
    for (int round = 0; round < 8; ++round) {
      std::vector<long long> first(n_fields), count(n_fields);
      long long n = 0;
      for (int f = 0; f < n_fields; ++f) {
        first[f] = o.sample_offset + have[f];
        count[f] = std::max<long long>(0, want[f] - have[f]);
        n += count[f];
      }
      if (n == 0) break;
      run_round(first, count, pl);
      for (int f = 0; f < n_fields; ++f) have[f] += count[f];
      bool more = false;
      for (int f = 0; f < n_fields; ++f) {
        double mean, var;
        plain_stats(f, &mean, &var);
        const long long need = (long long)std::ceil(1.15 * var / se2) + 1;
        // the control variate pays where the plain estimate would need well
        // more samples than the training set
        if (round == 0 && need >= std::max<long long>(cp.cv_threshold, 2LL * cp.M_train)) is_cv[f] = 1;
        if (is_cv[f]) {
          want[f] = std::min<long long>({std::max<long long>(have[f], cp.M_train), M_max, 4 * have[f]});
        } else if (var / (double)have[f] <= se2 || have[f] >= M_max) {
          want[f] = have[f];
        } else {
          want[f] = std::min<long long>({M_max, std::max<long long>(need, have[f] + 1), 4 * have[f]});
        }
        more = more || want[f] > have[f];
      }
      if (!more) break;
    }
    // 2. train on every plain sample of the control-variate fields
    std::vector<double> tB, tphi;
    std::vector<long long> ts;
    for (int f = 0; f < n_fields; ++f)
      if (is_cv[f])
        for (long long i = 0; i < have[f]; ++i) {
          tB.push_back(fields[f]);
          ts.push_back(o.sample_offset + i);
          tphi.push_back(pl[f][3 * i]);
        }
    std::vector<double> mu(n_fields, 0.0), vmu(n_fields, 0.0);
    double cv_ms = 0.0;  // host wall time of the control-variate work (rp_stats.cv_ms)
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto ms_since = [](std::chrono::steady_clock::time_point t0) {
      return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    };
    const auto t_train = now();
    if (tB.size() >= 2) {
      rp_cv_options net = cp.net;
      net.stream = o.stream;
      rp_status cs = rp_cv_create(sys, &net, &cv);
      if (cs != RP_OK) return cs;
      cs = rp_cv_train(cv, (int)tB.size(), tB.data(), ts.data(), seed, o.pair_id, tphi.data(), nullptr);
      if (cs != RP_OK) return cs;
      std::vector<double> Bcv;
      std::vector<int> fidx;
      for (int f = 0; f < n_fields; ++f)
        if (is_cv[f]) {
          Bcv.push_back(fields[f]);
          fidx.push_back(f);
        }
      std::vector<double> m(Bcv.size()), vm(Bcv.size());
      // mu from its own directions (pair word with bit 30 set)
      cs = rp_cv_mean(cv, (int)Bcv.size(), Bcv.data(), cp.n_mc, seed, o.pair_id ^ 0x40000000u,
                      m.data(), vm.data());
      if (cs != RP_OK) return cs;
      for (size_t i = 0; i < fidx.size(); ++i) {
        mu[fidx[i]] = m[i];
        vmu[fidx[i]] = vm[i];
      }
    } else {
      std::fill(is_cv.begin(), is_cv.end(), 0);
    }
    cv_ms += ms_since(t_train);
    // 3. control-variate rounds on fresh samples until the combined SE meets the target
    std::vector<double> cvout(5 * (size_t)n_fields, 0.0);
    auto cv_estimates = [&]() {
      std::vector<long long> off, cnt;
      std::vector<double> allp, allg;
      std::vector<int> fidx;
      for (int f = 0; f < n_fields; ++f)
        if (is_cv[f] && have_cv[f] >= 2) {
          off.push_back((long long)allg.size());
          cnt.push_back(have_cv[f]);
          allp.insert(allp.end(), cvs[f].begin(), cvs[f].end());
          allg.insert(allg.end(), cvg[f].begin(), cvg[f].end());
          fidx.push_back(f);
        }
      if (fidx.empty()) return;
      std::vector<double> m(fidx.size()), vm(fidx.size()), o5(5 * fidx.size());
      for (size_t i = 0; i < fidx.size(); ++i) {
        m[i] = mu[fidx[i]];
        vm[i] = vmu[fidx[i]];
      }
      rp_status cs = rp_cv_estimate(cv, (int)fidx.size(), off.data(), cnt.data(), allp.data(),
                                    allg.data(), m.data(), vm.data(), o5.data());
      if (cs != RP_OK) throw CudaFail{cs, rp_last_error()};
      for (size_t i = 0; i < fidx.size(); ++i)
        for (int q = 0; q < 5; ++q) cvout[5 * fidx[i] + q] = o5[5 * i + q];
    };
    std::vector<long long> want_cv(n_fields, 0);
    for (int f = 0; f < n_fields; ++f)
      if (is_cv[f]) {
        double mean, var;
        plain_stats(f, &mean, &var);
        const double rem = 1.0 / se2 - (double)have[f] / var;  // precision still missing
        want_cv[f] = rem > 0 ? std::max<long long>(16, (long long)std::ceil(0.3 * var * rem)) : 0;
      }
    for (int round = 0; round < 8; ++round) {
      std::vector<long long> first(n_fields), count(n_fields);
      long long n = 0;
      for (int f = 0; f < n_fields; ++f) {
        first[f] = kCvBase + o.sample_offset + have_cv[f];
        count[f] = is_cv[f] ? std::max<long long>(0, want_cv[f] - have_cv[f]) : 0;
        n += count[f];
      }
      if (n == 0) break;
      std::vector<std::vector<double>> fresh(n_fields);
      run_round(first, count, fresh);
      for (int f = 0; f < n_fields; ++f) {
        if (!count[f]) continue;
        std::vector<double> Bf(count[f], fields[f]), g(count[f]);
        std::vector<long long> sf(count[f]);
        for (long long i = 0; i < count[f]; ++i) sf[i] = first[f] + i;
        const auto t_eval = now();
        rp_status cs = rp_cv_eval(cv, (int)count[f], Bf.data(), sf.data(), seed, o.pair_id, g.data());
        cv_ms += ms_since(t_eval);
        if (cs != RP_OK) return cs;
        cvs[f].insert(cvs[f].end(), fresh[f].begin(), fresh[f].end());
        cvg[f].insert(cvg[f].end(), g.begin(), g.end());
        have_cv[f] += count[f];
      }
      const auto t_est = now();
      cv_estimates();
      cv_ms += ms_since(t_est);
      bool more = false;
      for (int f = 0; f < n_fields; ++f) {
        if (!is_cv[f] || have_cv[f] < 2) continue;
        double mean, var;
        plain_stats(f, &mean, &var);
        const double prec = (double)have[f] / var + 1.0 / (cvout[5 * f + 1] * cvout[5 * f + 1]);
        if (prec >= 1.0 / se2 || have_cv[f] >= M_max) continue;
        // residual variance per control-variate sample
        const double vres = cvout[5 * f + 1] * cvout[5 * f + 1] * (double)have_cv[f];
        const double need = std::ceil(1.15 * vres * (1.0 / se2 - (double)have[f] / var)) + 1;
        want_cv[f] = std::min<long long>({M_max, std::max<long long>((long long)need, have_cv[f] + 1),
                                          4 * have_cv[f]});
        more = true;
      }
      if (!more) break;
    }
    // 4. plain statistics on the device over every plain sample, then combine
    long long tot = 0;
    std::vector<long long> offcnt(2 * (size_t)n_fields);
    for (int f = 0; f < n_fields; ++f) {
      offcnt[f] = tot;
      offcnt[n_fields + f] = have[f];
      tot += have[f];
    }
    std::vector<double> all;
    all.reserve((size_t)tot * 3);
    for (int f = 0; f < n_fields; ++f) all.insert(all.end(), pl[f].begin(), pl[f].end());
    double* d_all = ar.get<double>((size_t)std::max<long long>(tot, 1) * 3);
    long long* d_off = ar.get<long long>(2 * (size_t)n_fields);
    double* d_stats = ar.get<double>((size_t)n_fields * 5);
    ck(cudaMemcpyAsync(d_all, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice, st), "h2d");
    ck(cudaMemcpyAsync(d_off, offcnt.data(), offcnt.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
    eng.h2d += (long long)(all.size() * sizeof(double) + offcnt.size() * sizeof(long long));
    ck(rp::launch_stats(d_all, d_off, d_off + n_fields, n_fields, d_stats, st), "stats kernel");
    eng.launches++;
    std::vector<double> pst((size_t)n_fields * 5);
    ck(cudaMemcpyAsync(pst.data(), d_stats, pst.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h stats");
    d2h += (long long)pst.size() * sizeof(double);
    ck(cudaEventRecord(ev.b, st), "cudaEventRecord");
    ck(cudaStreamSynchronize(st), "kernel execution");
    for (int f = 0; f < n_fields; ++f) {
      const double mp = pst[5 * f], sp = pst[5 * f + 2];
      double* of = out + 8 * f;
      of[2] = mp;
      of[3] = sp;
      if (is_cv[f] && have_cv[f] >= 2) {
        const double mc = cvout[5 * f], sc = cvout[5 * f + 1];
        const double wp = sp > 0 ? 1.0 / (sp * sp) : 0.0, wc = sc > 0 ? 1.0 / (sc * sc) : 0.0;
        of[0] = (wp + wc) > 0 ? (wp * mp + wc * mc) / (wp + wc) : mp;
        of[1] = (wp + wc) > 0 ? 1.0 / std::sqrt(wp + wc) : sp;
        of[4] = mc;
        of[5] = sc;
        of[6] = cvout[5 * f + 4];
        of[7] = 1.0;
      } else {
        of[0] = mp;
        of[1] = sp;
        of[4] = of[5] = of[6] = of[7] = 0.0;
      }
      if (M_plain) M_plain[f] = (int)have[f];
      if (M_cv) M_cv[f] = (int)have_cv[f];
    }
    fill_stats(stats, eng, total_items, R, n_c, ev.a, ev.b, o.profile != 0, d2h);
    if (stats) stats->cv_ms = cv_ms;
  }
  ck(cudaStreamSynchronize(st), "free");
  return RP_OK;
}

// Several radical pairs in one pass (see rp_yields_batch in rp.h): systems are
// grouped by size so that a row slot is at most twice a system's Z; every
// group runs all its (system, field, sample) items on one pool of rows.
template <typename T>
rp_status run_batch(int n_sys, rp_system* const* systems, const int* n_fields,
                    const double* const* fields, const int* M, const double* t_max, uint64_t seed,
                    const rp_options& o, double* const* out, rp_stats* stats) {
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  const double tol = o.tol > 0 ? o.tol : default_tol(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  // plans and per-sample output offsets of every (system, field)
  std::vector<std::vector<rp::FieldPlan>> plans(n_sys);
  std::vector<long long> base(n_sys + 1, 0);
  long long n_pairs = 0;
  for (int s = 0; s < n_sys; ++s) {
    rp_status ps = plan_all(systems[s]->hs, n_fields[s], fields[s], t_max[s], n_c, tol, plans[s]);
    if (ps != RP_OK) return fail(ps, "system " + std::to_string(s) + ": " + rp_last_error());
    base[s + 1] = base[s] + (long long)n_fields[s] * M[s];
    n_pairs += n_fields[s];
  }
  const long long n_samples = base[n_sys];
  // groups by ceil(log2 Z), largest first
  std::vector<int> order(n_sys);
  for (int s = 0; s < n_sys; ++s) order[s] = s;
  auto lg = [&](int s) {
    int b = 0;
    while ((1LL << b) < systems[s]->hs.Z) ++b;
    return b;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return lg(a) > lg(b); });
  EventPair ev;
  long long launches = 0, step_launches = 0, row_terms = 0, h2d = 0, d2h = 0, graphs = 0;
  double step_bytes = 0.0, step_ms = 0.0;
  long long step_timed = 0;
  int R_max = 0;
  Arena outer(st);
  double* d_ps = outer.get<double>((size_t)std::max<long long>(n_samples, 1) * 3);
  ck(cudaEventRecord(ev.a, st), "cudaEventRecord");
  for (size_t g0 = 0; g0 < order.size();) {
    size_t g1 = g0;
    while (g1 < order.size() && lg(order[g1]) == lg(order[g0])) ++g1;
    std::vector<const rp::HostSystem*> group;
    std::vector<uint32_t> pairs;
    std::vector<rp::FieldPlan> gplans;
    std::vector<int> sys_of_field;
    std::vector<long long> first, count, out0;
    for (size_t i = g0; i < g1; ++i) {
      const int s = order[i];
      const int gs = (int)group.size();
      group.push_back(&systems[s]->hs);
      pairs.push_back(o.pair_id + (uint32_t)s);
      for (int f = 0; f < n_fields[s]; ++f) {
        gplans.push_back(plans[s][f]);
        sys_of_field.push_back(gs);
        first.push_back(0);
        count.push_back(M[s]);
        out0.push_back(base[s] + (long long)f * M[s]);
      }
    }
    const std::vector<Item> items = make_items(gplans, first, count, out0, o.sample_offset, SampleMode{},
                                               &sys_of_field);
    {
      Arena ar(st);
      YieldEngine<T> eng(group, o, n_c, st, ar, &pairs);
      eng.set_seed(seed);
      eng.set_fields(gplans);
      long long Zmax = 1;
      for (auto* h : group) Zmax = std::max<long long>(Zmax, h->Z);
      rp::HostSystem probe;
      probe.Z = Zmax;
      const int R = choose_rows<T>(probe, o, n_c, (long long)items.size());
      R_max = std::max(R_max, R);
      eng.alloc_rows(R);
      eng.run(items, d_ps);
      ck(cudaStreamSynchronize(st), "group");
      launches += eng.launches;
      graphs += eng.graph_launches;
      step_launches += eng.step_launches;
      row_terms += eng.row_terms;
      h2d += eng.h2d;
      d2h += eng.d2h;
      step_bytes += eng.step_bytes_all;
      for (size_t i = 0; i + 1 < eng.pev.size(); i += 2) {
        float t = 0.f;
        ck(cudaEventElapsedTime(&t, eng.pev[i], eng.pev[i + 1]), "cudaEventElapsedTime");
        step_ms += t;
        step_timed += eng.pev_launches[i / 2];
      }
    }
    g0 = g1;
  }
  // per-(system, field) statistics on the device
  std::vector<long long> offcnt(2 * (size_t)n_pairs);
  {
    long long q = 0;
    for (int s = 0; s < n_sys; ++s)
      for (int f = 0; f < n_fields[s]; ++f, ++q) {
        offcnt[q] = base[s] + (long long)f * M[s];
        offcnt[n_pairs + q] = M[s];
      }
  }
  long long* d_off = outer.get<long long>(2 * (size_t)n_pairs);
  double* d_stats = outer.get<double>(5 * (size_t)n_pairs);
  ck(cudaMemcpyAsync(d_off, offcnt.data(), offcnt.size() * sizeof(long long), cudaMemcpyHostToDevice, st), "h2d");
  h2d += (long long)(offcnt.size() * sizeof(long long));
  ck(rp::launch_stats(d_ps, d_off, d_off + n_pairs, (int)n_pairs, d_stats, st), "stats kernel");
  ++launches;
  std::vector<double> hst(5 * (size_t)n_pairs);
  ck(cudaMemcpyAsync(hst.data(), d_stats, hst.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
  d2h += (long long)(hst.size() * sizeof(double));
  ck(cudaEventRecord(ev.b, st), "cudaEventRecord");
  ck(cudaStreamSynchronize(st), "batch");
  {
    long long q = 0;
    for (int s = 0; s < n_sys; ++s)
      for (int f = 0; f < n_fields[s]; ++f, ++q)
        for (int c = 0; c < 5; ++c) out[s][5 * f + c] = hst[5 * q + c];
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->kernel_launches = launches;
    stats->step_launches = step_launches;
    stats->row_terms = row_terms;
    stats->propagations = n_samples;
    stats->rows = R_max;
    stats->n_cheb = n_c;
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, ev.a, ev.b), "cudaEventElapsedTime");
    stats->device_ms = ms;
    stats->step_ms = step_ms;
    stats->step_bytes = step_bytes;
    stats->step_launches_timed = step_timed;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
    stats->graph_launches = graphs;
  }
  return RP_OK;
}

}  // namespace

namespace rp {
void set_last_error(const std::string& msg) { g_err = msg; }
// Device allocation through the caller's hooks (rp_set_allocator) or
// cudaMallocAsync; throws nothing, returns NULL on failure.
void* device_alloc(size_t bytes, cudaStream_t st) {
  try {
    return dev_alloc(bytes, st);
  } catch (const CudaFail&) {
    return nullptr;
  }
}
void device_free(void* p, cudaStream_t st) { dev_free(p, st); }
rp_status device_check() { return check_device(); }
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

rp_status rp_rotate(const rp_system* s, double theta, double phi, rp_system** out) {
  g_err.clear();
  if (!s || !out) return fail(RP_EINVAL, "system or out is NULL");
  if (!std::isfinite(theta) || !std::isfinite(phi)) return fail(RP_EINVAL, "non-finite angle");
  const rp::HostSystem& h = s->hs;
  // R = R_y(-theta) R_z(-phi) takes n(theta, phi) to z; tensors A' = R A R^T
  const double ct = std::cos(theta), st = std::sin(theta), cp = std::cos(phi), sp = std::sin(phi);
  const double Rz[3][3] = {{cp, sp, 0.0}, {-sp, cp, 0.0}, {0.0, 0.0, 1.0}};
  const double Ry[3][3] = {{ct, 0.0, -st}, {0.0, 1.0, 0.0}, {st, 0.0, ct}};
  double Rm[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Rm[i][j] = 0.0;
      for (int q = 0; q < 3; ++q) Rm[i][j] += Ry[i][q] * Rz[q][j];
    }
  std::vector<double> A2((size_t)9 * h.n_nuc);
  for (int k = 0; k < h.n_nuc; ++k) {
    const double* A = &h.A[9 * k];
    double* B = &A2[9 * (size_t)k];
    const bool iso = A[1] == 0.0 && A[2] == 0.0 && A[3] == 0.0 && A[5] == 0.0 && A[6] == 0.0 &&
                     A[7] == 0.0 && A[0] == A[4] && A[0] == A[8];
    if (iso) {  // a multiple of the identity is invariant
      for (int q = 0; q < 9; ++q) B[q] = A[q];
      continue;
    }
    double T[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        T[i][j] = 0.0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) T[i][j] += Rm[i][p] * A[3 * p + q] * Rm[j][q];
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) B[3 * i + j] = 0.5 * (T[i][j] + T[j][i]);
  }
  return rp_create(h.n_nuc, h.radical.data(), h.two_I.data(), A2.data(), h.k_S, h.k_T, h.J_mT, out);
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
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic < 0 || o.deterministic > 3) return fail(RP_EINVAL, "deterministic must be 0, 1, 2 or 3");
  if (o.deterministic == 3 && s->hs.aniso)
    return fail(RP_EINVAL, "the J_z-sector trace (deterministic = 3) needs isotropic hyperfine couplings");
  if ((o.deterministic == 0 || o.deterministic == 2) && M < 2)
    return fail(RP_EINVAL, "M must be >= 2 (the standard error needs it)");
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

rp_status rp_basis_indices(uint64_t seed, uint32_t pair_id, long long sample_offset, int M,
                           long long Z, long long* out) {
  g_err.clear();
  if (M < 0 || Z < 1 || sample_offset < 0) return fail(RP_EINVAL, "need M >= 0, Z >= 1, sample_offset >= 0");
  if (M > 0 && !out) return fail(RP_EINVAL, "out is NULL");
  for (int i = 0; i < M; ++i) out[i] = rp::basis_draw(seed, pair_id, sample_offset + i, Z);
  return RP_OK;
}

rp_status rp_field_sums(int n_fields, const double* out, long long M, double* sums) {
  g_err.clear();
  if (n_fields < 0 || (n_fields > 0 && (!out || !sums))) return fail(RP_EINVAL, "bad arguments");
  if (M < 2) return fail(RP_EINVAL, "M must be >= 2 (the standard error needs it)");
  const double m = (double)M;
  for (int f = 0; f < n_fields; ++f) {
    const double* o = out + 5 * (size_t)f;
    double* s = sums + 5 * (size_t)f;
    // sample variance s^2 = M SE^2 (Eq. 23, M - 1), sum x^2 = (M - 1) s^2 + M mean^2
    s[0] = m * o[0];
    s[1] = (m - 1.0) * m * o[2] * o[2] + m * o[0] * o[0];
    s[2] = m * o[1];
    s[3] = (m - 1.0) * m * o[3] * o[3] + m * o[1] * o[1];
    s[4] = m * o[4];
  }
  return RP_OK;
}

rp_status rp_combine_sums(int n_fields, const double* sums, long long M, double* out) {
  g_err.clear();
  if (n_fields < 0 || (n_fields > 0 && (!out || !sums))) return fail(RP_EINVAL, "bad arguments");
  if (M < 2) return fail(RP_EINVAL, "M must be >= 2");
  const double m = (double)M;
  for (int f = 0; f < n_fields; ++f) {
    const double* s = sums + 5 * (size_t)f;
    double* o = out + 5 * (size_t)f;
    const double ms = s[0] / m, mt = s[2] / m;
    const double vs = std::max(s[1] - m * ms * ms, 0.0) / (m - 1.0);
    const double vt = std::max(s[3] - m * mt * mt, 0.0) / (m - 1.0);
    o[0] = ms;
    o[1] = mt;
    o[2] = std::sqrt(vs / m);
    o[3] = std::sqrt(vt / m);
    o[4] = s[4] / m;
  }
  return RP_OK;
}

rp_status rp_trace_propagations(const rp_system* s, int deterministic, long long* n) {
  g_err.clear();
  if (!s || !n) return fail(RP_EINVAL, "system or n is NULL");
  if (deterministic == 1) {
    *n = s->hs.Z;
    return RP_OK;
  }
  if (deterministic != 3) return fail(RP_EINVAL, "deterministic must be 1 or 3");
  if (s->hs.aniso)
    return fail(RP_EINVAL, "the J_z-sector trace (deterministic = 3) needs isotropic hyperfine couplings");
  try {
    std::vector<int> rank, n_of;
    *n = rp::sector_table(s->hs, &rank, &n_of);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
  return RP_OK;
}

rp_status rp_time_trace(rp_system* s, double B, int M, uint64_t seed, double t_max,
                        const rp_options* opt, int max_times, int* n_times, double* t,
                        double* out) {
  g_err.clear();
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (!s || !n_times) return fail(RP_EINVAL, "system or n_times is NULL");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic == 3) return fail(RP_ENOTIMPL, "rp_time_trace does not take the J_z-sector trace (deterministic = 3)");
  if (o.deterministic < 0 || o.deterministic > 2) return fail(RP_EINVAL, "deterministic must be 0, 1 or 2");
  if (o.deterministic != 1 && M < 1) return fail(RP_EINVAL, "M must be >= 1");
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return fail(RP_EINVAL, "t_max must be positive and finite");
  if (!std::isfinite(B)) return fail(RP_EINVAL, "non-finite field");
  if (o.sample_offset < 0) return fail(RP_EINVAL, "sample_offset must be >= 0");
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  try {
    std::vector<rp::FieldPlan> plans;
    rp_status ps = plan_all(s->hs, 1, &B, t_max, n_c, o.tol > 0 ? o.tol : default_tol(o.precision),
                            plans);
    if (ps != RP_OK) return ps;
    if (plans[0].n_macro + 1 > (long long)INT32_MAX) return fail(RP_EINVAL, "too many time points");
    const int nt = (int)(plans[0].n_macro + 1);
    *n_times = nt;
    if (!t || !out) return RP_OK;  // size query
    if (max_times < nt) return fail(RP_EINVAL, "max_times is smaller than the number of time points");
    rp_status ds = check_device();
    if (ds != RP_OK) return ds;
    if (o.precision == RP_FP64) return run_time_trace<double>(s, B, M, seed, t_max, o, nt, t, out);
    return run_time_trace<float>(s, B, M, seed, t_max, o, nt, t, out);
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
}

rp_status rp_time_observable(rp_system* s, double B, int M, uint64_t seed, double t_max,
                             const rp_options* opt, const double* A, int max_times,
                             int* n_times, double* t, double* out) {
  g_err.clear();
  if (!A) return fail(RP_EINVAL, "A is NULL");
  for (int q = 0; q < 32; ++q)
    if (!std::isfinite(A[q])) return fail(RP_EINVAL, "non-finite operator entry");
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (!s || !n_times) return fail(RP_EINVAL, "system or n_times is NULL");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic == 3) return fail(RP_ENOTIMPL, "rp_time_observable does not take the J_z-sector trace (deterministic = 3)");
  if (o.deterministic < 0 || o.deterministic > 2) return fail(RP_EINVAL, "deterministic must be 0, 1 or 2");
  if (o.deterministic != 1 && M < 1) return fail(RP_EINVAL, "M must be >= 1");
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return fail(RP_EINVAL, "t_max must be positive and finite");
  if (!std::isfinite(B)) return fail(RP_EINVAL, "non-finite field");
  if (o.sample_offset < 0) return fail(RP_EINVAL, "sample_offset must be >= 0");
  const int n_c = o.n_cheb > 0 ? o.n_cheb : default_ncheb(o.precision);
  if (n_c % 4 != 0 || n_c < 8 || n_c > 88)
    return fail(RP_EINVAL, "n_cheb must be a multiple of 4 in [8, 88]");
  try {
    std::vector<rp::FieldPlan> plans;
    rp_status ps = plan_all(s->hs, 1, &B, t_max, n_c, o.tol > 0 ? o.tol : default_tol(o.precision),
                            plans);
    if (ps != RP_OK) return ps;
    if (plans[0].n_macro + 1 > (long long)INT32_MAX) return fail(RP_EINVAL, "too many time points");
    const int nt = (int)(plans[0].n_macro + 1);
    *n_times = nt;
    if (!t || !out) return RP_OK;  // size query
    if (max_times < nt) return fail(RP_EINVAL, "max_times is smaller than the number of time points");
    rp_status ds = check_device();
    if (ds != RP_OK) return ds;
    if (o.precision == RP_FP64)
      return run_time_trace<double>(s, B, M, seed, t_max, o, nt, t, nullptr, A, out);
    return run_time_trace<float>(s, B, M, seed, t_max, o, nt, t, nullptr, A, out);
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
}

rp_status rp_yields_converged(rp_system* s, int n_fields, const double* fields, double se_target,
                              int M_min, int M_max, uint64_t seed, double t_max,
                              const rp_options* opt, double* out, int* M_used, rp_stats* stats) {
  g_err.clear();
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (n_fields < 0) return fail(RP_EINVAL, "n_fields must be >= 0");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic) return fail(RP_EINVAL, "rp_yields_converged samples coherent states only");
  if (!(se_target > 0.0) || !std::isfinite(se_target)) return fail(RP_EINVAL, "se_target must be positive");
  if (M_min < 2 || M_max < M_min) return fail(RP_EINVAL, "need 2 <= M_min <= M_max");
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
      return run_converged<double>(s, n_fields, fields, se_target, M_min, M_max, seed, t_max, o,
                                   out, M_used, stats);
    return run_converged<float>(s, n_fields, fields, se_target, M_min, M_max, seed, t_max, o, out,
                                M_used, stats);
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
}

void rp_cv_default_plan(rp_cv_plan* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->M_train = 300;
  p->cv_threshold = 150;
  p->n_mc = 1LL << 18;
  rp_cv_default_options(&p->net);
}

rp_status rp_yields_cv(rp_system* s, int n_fields, const double* fields, double se_target,
                       int M_min, int M_max, uint64_t seed, double t_max, const rp_options* opt,
                       const rp_cv_plan* plan, double* out, int* M_plain, int* M_cv,
                       rp_stats* stats) {
  g_err.clear();
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  rp_cv_plan cp;
  if (plan) cp = *plan;
  else rp_cv_default_plan(&cp);
  if (!s) return fail(RP_EINVAL, "system is NULL");
  if (n_fields < 0) return fail(RP_EINVAL, "n_fields must be >= 0");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic) return fail(RP_EINVAL, "rp_yields_cv samples coherent states only");
  if (!(se_target > 0.0) || !std::isfinite(se_target)) return fail(RP_EINVAL, "se_target must be positive");
  if (M_min < 2 || M_max < M_min) return fail(RP_EINVAL, "need 2 <= M_min <= M_max");
  if (cp.M_train < 2 || cp.cv_threshold < 2 || cp.n_mc < 2) return fail(RP_EINVAL, "bad control-variate plan");
  if (!(t_max > 0.0) || !std::isfinite(t_max)) return fail(RP_EINVAL, "t_max must be positive and finite");
  if (o.sample_offset < 0 || o.sample_offset >= (1LL << 39)) return fail(RP_EINVAL, "sample_offset must be in [0, 2^39)");
  if (n_fields > 0 && (!fields || !out)) return fail(RP_EINVAL, "NULL fields or out");
  for (int f = 0; f < n_fields; ++f)
    if (!std::isfinite(fields[f])) return fail(RP_EINVAL, "non-finite field");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_fields == 0) return RP_OK;
  rp_status ds = check_device();
  if (ds != RP_OK) return ds;
  try {
    if (o.precision == RP_FP64)
      return run_converged_cv<double>(s, n_fields, fields, se_target, M_min, M_max, seed, t_max, o,
                                      cp, out, M_plain, M_cv, stats);
    return run_converged_cv<float>(s, n_fields, fields, se_target, M_min, M_max, seed, t_max, o, cp,
                                   out, M_plain, M_cv, stats);
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(RP_ENOMEM, "host allocation failed");
  }
}

rp_status rp_yields_batch(int n_sys, rp_system* const* systems, const int* n_fields,
                          const double* const* fields, const int* M, const double* t_max,
                          uint64_t seed, const rp_options* opt, double* const* out,
                          rp_stats* stats) {
  g_err.clear();
  rp_options o;
  if (opt) o = *opt;
  else rp_default_options(&o);
  if (n_sys < 0) return fail(RP_EINVAL, "n_sys must be >= 0");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n_sys == 0) return RP_OK;
  if (!systems || !n_fields || !fields || !M || !t_max || !out) return fail(RP_EINVAL, "NULL argument");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return fail(RP_EINVAL, "bad precision");
  if (bad_kernel_choice(o)) return fail(RP_EINVAL, "kernel must be 0..5, gram 0..2 and graph 0 or 1");
  if (o.deterministic) return fail(RP_EINVAL, "rp_yields_batch samples coherent states only");
  if (o.sample_offset < 0) return fail(RP_EINVAL, "sample_offset must be >= 0");
  long long total = 0;
  for (int s = 0; s < n_sys; ++s) {
    const std::string w = "system " + std::to_string(s) + ": ";
    if (!systems[s]) return fail(RP_EINVAL, w + "NULL system");
    if (n_fields[s] < 0) return fail(RP_EINVAL, w + "n_fields must be >= 0");
    if (n_fields[s] > 0 && (!fields[s] || !out[s])) return fail(RP_EINVAL, w + "NULL fields or out");
    if (M[s] < 2) return fail(RP_EINVAL, w + "M must be >= 2");
    if (!(t_max[s] > 0.0) || !std::isfinite(t_max[s])) return fail(RP_EINVAL, w + "t_max must be positive and finite");
    for (int f = 0; f < n_fields[s]; ++f)
      if (!std::isfinite(fields[s][f])) return fail(RP_EINVAL, w + "non-finite field");
    total += (long long)n_fields[s] * M[s];
  }
  if (total == 0) return RP_OK;
  rp_status ds = check_device();
  if (ds != RP_OK) return ds;
  try {
    if (o.precision == RP_FP64)
      return run_batch<double>(n_sys, systems, n_fields, fields, M, t_max, seed, o, out, stats);
    return run_batch<float>(n_sys, systems, n_fields, fields, M, t_max, seed, o, out, stats);
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
      const rp::HamDev<double> H = make_ham<double>(hs);
      auto* d = ar.get<rp::FieldDev<double>>(1);
      auto* dh = ar.get<rp::HamDev<double>>(1);
      ck(cudaMemcpyAsync(d, &F, sizeof(F), cudaMemcpyHostToDevice, st), "h2d");
      ck(cudaMemcpyAsync(dh, &H, sizeof(H), cudaMemcpyHostToDevice, st), "h2d");
      const rp::SysTab<double> S{dh, nullptr, nullptr, nullptr, hs.Z, 0, nullptr};
      ck(rp::launch_step<double>(S, &H, H.aniso, 1, d, nullptr, nullptr, 0, nullptr, n_vec, (const double*)x,
                                 nullptr, (double*)y, nullptr, nullptr, nullptr, 0, 0,
                                 rp::MODE_APPLY, 0, st), "apply kernel");
    } else {
      rp::FieldDev<float> F{(float)(rp::kGammaE * B), 1.f, 0.f, (float)(0.5 * kbar)};
      const rp::HamDev<float> H = make_ham<float>(hs);
      auto* d = ar.get<rp::FieldDev<float>>(1);
      auto* dh = ar.get<rp::HamDev<float>>(1);
      ck(cudaMemcpyAsync(d, &F, sizeof(F), cudaMemcpyHostToDevice, st), "h2d");
      ck(cudaMemcpyAsync(dh, &H, sizeof(H), cudaMemcpyHostToDevice, st), "h2d");
      const rp::SysTab<float> S{dh, nullptr, nullptr, nullptr, hs.Z, 0, nullptr};
      ck(rp::launch_step<float>(S, &H, H.aniso, 1, d, nullptr, nullptr, 0, nullptr, n_vec, (const float*)x, nullptr,
                                (float*)y, nullptr, nullptr, nullptr, 0, 0, rp::MODE_APPLY, 0, st),
         "apply kernel");
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
    auto* dl = ar.get<rp::LayoutDev>(1);
    ck(cudaMemcpyAsync(dl, &L, sizeof(L), cudaMemcpyHostToDevice, st), "h2d");
    if (precision == RP_FP64) {
      const rp::SysTab<double> S{nullptr, dl, nullptr, nullptr, hs.Z, pair_id, nullptr};
      ck(rp::launch_coherent_amps<double>(S, d_s, nullptr, n, seed, amps, uv, st), "coherent amplitudes");
      ck(rp::launch_init_state<double>(S, amps, d_s, nullptr, nullptr, n, 0, (double*)psi,
                                       (double*)psi, nullptr, nullptr, st), "initial states");
    } else {
      const rp::SysTab<float> S{nullptr, dl, nullptr, nullptr, hs.Z, pair_id, nullptr};
      ck(rp::launch_coherent_amps<float>(S, d_s, nullptr, n, seed, amps, uv, st), "coherent amplitudes");
      ck(rp::launch_init_state<float>(S, amps, d_s, nullptr, nullptr, n, 0, (float*)psi,
                                      (float*)psi, nullptr, nullptr, st), "initial states");
    }
    if (angles && hs.n_nuc > 0)
      ck(cudaMemcpyAsync(angles, uv, (size_t)n * hs.n_nuc * 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "d2h");
    ck(cudaStreamSynchronize(st), "init kernels");
  } catch (const CudaFail& e) {
    return fail(e.st, e.msg);
  }
  return RP_OK;
}

}  // extern "C"
