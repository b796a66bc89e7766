// rp_tune: measured choice of the launch configuration of rp_yields.
//
// The knobs are the ones that change how the same propagation is executed,
// never what it computes (Eqs. 20, 22 are evaluated to the same tolerance by
// every candidate):
//   kernel  1 = one launch per Chebyshev term, 3 = the same with the partner
//           tiles staged by bulk copies (where the layout allows), 2 = a whole
//           macro-step per launch with the row in shared memory (only where
//           Z fits), 4 = a whole macro-step per launch with the row in the
//           distributed shared memory of a thread-block cluster (FP32
//           isotropic systems that fit), 5 = one persistent launch over all
//           propagations (only where Z fits one CTA; graph has no effect);
//   n_cheb  terms per macro-step (the planner then picks the step h that
//           meets the tolerance: more terms, longer steps, a larger
//           n_cheb x n_cheb time-integral Gram and more singlet slices);
//   graph   eager launches or CUDA-graph replay of each macro-step.
// Each candidate propagates `rows` samples at one field over a few
// macro-steps through rp_yields (one untimed run, then the faster of two
// timed runs by the call's own CUDA events); the figure of merit is
// propagated sample-microseconds per second of device time, which compares
// candidates with different step lengths fairly.
//
// Results can be kept in a plain-text cache (one line per key: the device,
// precision, the system's spin multiset, anisotropy, Z, rows and field) whose
// path is given by the RP_TUNE_CACHE environment variable; without it every
// call measures.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/rp.h"
#include "rp_plan.h"

struct rp_system {
  rp::HostSystem hs;
};

namespace rp {
void set_last_error(const std::string& msg);  // rp_api.cu: message of rp_last_error()
}

namespace {

rp_status tfail(rp_status s, const std::string& m) {
  rp::set_last_error(m);
  return s;
}

std::mutex g_cache_mu;

std::string cache_key(const rp_system* s, const rp_options& o, int rows, double B) {
  const rp::HostSystem& hs = s->hs;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceProp prop;
  std::memset(&prop, 0, sizeof(prop));
  cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (char& c : name)
    if (c == ' ') c = '_';
  std::vector<int> spins(hs.two_I);
  std::sort(spins.begin(), spins.end());
  std::ostringstream k;
  k << "dev=" << name << "/" << sms << " prec=" << o.precision << " spins=";
  for (size_t i = 0; i < spins.size(); ++i) k << (i ? "," : "") << spins[i];
  if (spins.empty()) k << "-";
  k << " aniso=" << (hs.aniso ? 1 : 0) << " Z=" << hs.Z << " rows=" << rows;
  char b[32];
  std::snprintf(b, sizeof(b), "%.3g", std::fabs(B));
  k << " B=" << b << " det=" << (o.deterministic ? 1 : 0);
  return k.str();
}

// Cached line: "<key>|kernel n_cheb graph rate"
bool cache_lookup(const char* path, const std::string& key, rp_tune_result* r) {
  std::ifstream f(path);
  if (!f) return false;
  std::string line;
  bool hit = false;
  while (std::getline(f, line)) {
    const size_t bar = line.rfind('|');
    if (bar == std::string::npos || line.compare(0, bar, key) != 0 || bar != key.size()) continue;
    std::istringstream v(line.substr(bar + 1));
    int kern = 0, nc = 0, g = 0;
    double rate = 0.0;
    if (v >> kern >> nc >> g >> rate) {
      r->kernel = kern;
      r->n_cheb = nc;
      r->graph = g;
      r->rate = rate;
      hit = true;  // the last matching line wins
    }
  }
  return hit;
}

void cache_store(const char* path, const std::string& key, const rp_tune_result& r) {
  std::ofstream f(path, std::ios::app);
  if (!f) return;  // an unwritable cache only costs re-measuring
  f << key << "|" << r.kernel << " " << r.n_cheb << " " << r.graph << " " << r.rate << "\n";
}

struct Cand {
  int kernel, n_cheb, graph;
};

}  // namespace

extern "C" {

rp_status rp_tune(rp_system* s, double B, int rows, const rp_options* base, rp_options* tuned,
                  rp_tune_result* res) {
  rp_options o;
  if (base) o = *base;
  else rp_default_options(&o);
  if (!s || !tuned) return tfail(RP_EINVAL, "system or tuned is NULL");
  if (rows < 2) return tfail(RP_EINVAL, "rows must be >= 2");
  if (!std::isfinite(B)) return tfail(RP_EINVAL, "non-finite field");
  if (o.precision != RP_FP64 && o.precision != RP_FP32) return tfail(RP_EINVAL, "bad precision");
  rp_tune_result r;
  std::memset(&r, 0, sizeof(r));
  const char* path = std::getenv("RP_TUNE_CACHE");
  std::string key;
  if (path && *path) {
    key = cache_key(s, o, rows, B);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (cache_lookup(path, key, &r)) {
      r.from_cache = 1;
      *tuned = o;
      tuned->kernel = r.kernel;
      tuned->n_cheb = r.n_cheb;
      tuned->graph = r.graph;
      tuned->max_rows = rows;
      if (res) *res = r;
      return RP_OK;
    }
  }
  const long long Z = s->hs.Z;
  const long long small_max = o.precision == RP_FP64 ? 1024 : 2048;
  const std::vector<int> ncs = {32, 48, 64, 88};
  std::vector<Cand> cands;
  // kernel 3 differs from 1 only where it stages partner tiles (FP32, >= 8 spin-1/2);
  // kernel 4 only where a row fits a thread-block cluster (FP32, isotropic)
  const bool staged = o.precision == RP_FP32 && s->hs.n_half >= 8;
  bool cluster_ok = false;
  int default_kernel = o.precision == RP_FP32
                           ? rp::default_kernel_fp32(s->hs, &cluster_ok)
                           : (Z <= small_max ? (rp::persistent_default(Z, 1) ? 5 : 2) : 1);
  if (default_kernel == 5 && o.graph) default_kernel = 2;  // kernel 0 with graph replay
  for (int nc : ncs)
    for (int g = 0; g <= 1; ++g) {
      cands.push_back({1, nc, g});
      if (Z <= small_max) cands.push_back({2, nc, g});
      if (Z <= small_max && g == 0) cands.push_back({5, nc, 0});
      if (staged) cands.push_back({3, nc, g});
      if (cluster_ok && Z > small_max) cands.push_back({4, nc, g});
    }
  const int kTrialMacro = 6;
  double best = -1.0, base_rate = -1.0;
  Cand bc = cands[0];
  for (const Cand& c : cands) {
    rp_options t = o;
    t.kernel = c.kernel;
    t.n_cheb = c.n_cheb;
    t.graph = c.graph;
    t.max_rows = rows;
    t.profile = 0;
    rp_field_plan p;
    rp_status e = rp_plan_field(s, B, 1.0, t.precision, t.n_cheb, t.tol, &p, nullptr, nullptr);
    if (e != RP_OK) return e;
    const double t_trial = p.h * kTrialMacro;
    std::vector<double> out(5);
    double ms = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
      rp_stats st;
      e = rp_yields(s, 1, &B, rows, 12345, t_trial, &t, out.data(), nullptr, &st);
      if (e != RP_OK) return e;
      if (rep > 0) ms = std::min(ms, st.device_ms);
    }
    const double rate = (double)rows * t_trial / (ms * 1e-3);
    r.candidates++;
    const bool is_base = c.kernel == (o.kernel ? o.kernel : default_kernel) &&
                         c.n_cheb == (o.n_cheb ? o.n_cheb : 88) &&
                         c.graph == o.graph;
    if (is_base) base_rate = rate;
    if (rate > best) {
      best = rate;
      bc = c;
    }
  }
  r.kernel = bc.kernel;
  r.n_cheb = bc.n_cheb;
  r.graph = bc.graph;
  r.rate = best;
  r.base_rate = base_rate;
  if (path && *path) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    cache_store(path, key, r);
  }
  *tuned = o;
  tuned->kernel = r.kernel;
  tuned->n_cheb = r.n_cheb;
  tuned->graph = r.graph;
  tuned->max_rows = rows;
  if (res) *res = r;
  return RP_OK;
}

}  // extern "C"
