// Host side of one Lanczos chain: device state, the operator schedule and the recursions.
// Included once per precision translation unit (double: plain FP64 path; float: FP32
// orbitals and FFTs with FP64 Lanczos scalars).
#pragma once
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <future>
#include <thread>
#include <array>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "ll.h"
#include "split.cuh"
#include "tcproj.cuh"
#include "xypair.cuh"

#include <type_traits>

namespace ll {

struct ChainBase {
  virtual ~ChainBase() {}
  virtual int create(const ll_system_desc* d, cudaStream_t st, std::string& err) = 0;
  // create() reusing the u_{vk}(r) grids of `donor`, a chain of the same ground state (same
  // precision, grid, k-points, bands, sphere(k) and u_k: checked by a hash of those inputs)
  virtual int create_shared(const ll_system_desc* d, cudaStream_t st, ChainBase* donor, std::string& err) = 0;
  virtual int lanczos(int n, double* beta, double* gamma, double* z, int* done, std::string& err) = 0;
  // asynchronous halves of lanczos(): queue n steps on the chain's stream / wait for them and
  // fetch every coefficient so far
  virtual int enqueue(int n, std::string& err) = 0;
  virtual int collect(double* beta, double* gamma, double* z, int* done, std::string& err) = 0;
  virtual int steps_queued() const = 0;
  // kind / m_total: LL_EXTRAP_* continuation of the m coefficients to m_total (Sec. 3.3)
  virtual int spectrum(int m, int kind, int m_total, const double* w_ev, int nw, double eta_ev, double* chi,
                       double* ei, double* e, std::string& err) = 0;
  virtual int steps() const = 0;
  // replay of captured steps on/off (on by default where the stream allows it)
  virtual void set_graphs(bool on) = 0;
  virtual int apply(int upper, const double* x, double* out, std::string& err) = 0;
  virtual int get_map(int* out, std::string& err) = 0;
  virtual int get_start(double* y, std::string& err) = 0;
  virtual size_t bytes() const = 0;
  virtual int profile(int enable, std::string& err) = 0;
  virtual int profile_read(double* ms, long long* launches, long long* total, std::string& err) = 0;
};

// Per-kernel-class device time, bracketed by CUDA events on the chain's stream while
// profiling is on; launch counts are kept always.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  int used = 0;
  std::vector<int> cls, ea, eb;
  long long launches[LL_NPROF] = {0}, total = 0;
  int mark(cudaStream_t st) {
    if (!on) return -1;
    if (used == (int)pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      pool.push_back(e);
    }
    cudaEventRecord(pool[used], st);
    return used++;
  }
  void span(int c, int a, int b) {
    if (a < 0 || b < 0) return;
    cls.push_back(c); ea.push_back(a); eb.push_back(b);
  }
  void count(int c, int n = 1) { launches[c] += n; total += n; }
  void reset() {
    used = 0; cls.clear(); ea.clear(); eb.clear();
    for (auto& l : launches) l = 0;
    total = 0;
  }
  ~Profiler() { for (auto e : pool) cudaEventDestroy(e); }
};

ChainBase* make_chain_f64();
ChainBase* make_chain_f32();
int footprint_bytes(const ll_system_desc* d, size_t* out, std::string& err);

#define LL_CK(call)                                                                    \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);                        \
      return (e_ == cudaErrorMemoryAllocation) ? LL_ENOMEM : LL_ECUDA;                 \
    }                                                                                  \
  } while (0)

// Column/row tables of one sphere family, built on the host from the Miller lists.
struct HostSphere {
  int nks = 0, npw_pad = 0, ncol_max = 0, nrow_max = 0;
  std::vector<int> npw, off, ncol, nrow, colstart;
  std::vector<int4> col, row;
};

static inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Every floating-point input of a system finite: a NaN or an infinity would pass into every
// coefficient of the chain without tripping the breakdown checks.  The array pointers and the
// sphere sizes npw_k, npw_kq must already be valid.
struct FiniteCheck { const double* p; long len; const char* what; bool device; bool large; };

// The floating-point input arrays of a descriptor, with where they live.
static inline std::vector<FiniteCheck> input_arrays(const ll_system_desc* d) {
  long sk = 0, sq = 0;
  for (int k = 0; k < d->nks; ++k) sk += d->npw_k[k], sq += d->npw_kq[k];
  const long n3 = (long)d->nfft * d->nfft * d->nfft, nb = d->nbnd, np = d->nproj;
  const bool dv = d->where == LL_WHERE_DEVICE;
  return {{&d->lattice[0][0], 9, "lattice", false, false},  {d->q_cart, 3, "q_cart", false, false},
          {d->kcart, 3L * d->nks, "kcart", false, false},    {d->u_k, 2 * nb * sk, "u_k", dv, true},
          {d->u_kq, 2 * nb * sq, "u_kq", dv, true},          {d->eps_k, (long)d->nks * nb, "eps_k", false, false},
          {d->vloc_r, n3, "vloc_r", dv, true},               {d->rho_r, n3, "rho_r", dv, true},
          {d->beta_kq, 2 * np * sq, "beta_kq", dv, true},   {d->dij, np, "dij", false, false},
          {d->occ_k, d->occ_k ? (long)d->nks * nb : 0, "occ_k", false, false},
          {d->occ_kq, (d->occ_k && d->occ_kq) ? (long)d->nks * nb : 0, "occ_kq", false, false},
          {d->eps_kq, (d->occ_k && d->eps_kq) ? (long)d->nks * nb : 0, "eps_kq", false, false}};
}

// large_on_host: check the large arrays here too (the request loop refuses a malformed job at
// submit); ll_create checks them on the device after they are uploaded.
static inline bool inputs_finite(const ll_system_desc* d, std::string& err, bool large_on_host = true) {
  for (const auto& a : input_arrays(d))
    if (!a.device && (large_on_host || !a.large))
      for (long i = 0; i < a.len; ++i)
      if (!std::isfinite(a.p[i])) {
        err = std::string("non-finite value in ") + a.what + " at index " + std::to_string(i);
        return false;
      }
  return true;
}

static inline bool build_sphere(int nks, const int* npw, const int* mil, int n, HostSphere& h, std::string& err) {
  h.nks = nks;
  h.npw.assign(npw, npw + nks);
  h.off.resize(nks + 1);
  h.off[0] = 0;
  int maxnpw = 1;
  for (int k = 0; k < nks; ++k) {
    if (npw[k] <= 0) { err = "empty plane-wave sphere"; return false; }
    h.off[k + 1] = h.off[k] + npw[k];
    maxnpw = std::max(maxnpw, npw[k]);
  }
  h.npw_pad = round_up(maxnpw, 4);
  std::vector<std::vector<int4>> cols(nks), rows(nks);
  std::vector<std::vector<int>> starts(nks);
  std::vector<const char*> kerr(nks, nullptr);
  // the tables of one sphere (independent per k: built on several host threads)
  auto one = [&](int k) -> const char* {
    const int* m = mil + 3L * h.off[k];
    int lo[3] = {m[0], m[1], m[2]}, hi[3] = {m[0], m[1], m[2]};
    for (int i = 0; i < npw[k]; ++i) {
      for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], m[3 * i + a]); hi[a] = std::max(hi[a], m[3 * i + a]); }
      if (i > 0) {
        const int* p = m + 3 * (i - 1);
        const int* q = m + 3 * i;
        const bool less = p[0] < q[0] || (p[0] == q[0] && (p[1] < q[1] || (p[1] == q[1] && p[2] < q[2])));
        if (!less) return "Miller indices of a sphere are not strictly lexicographic";
      }
    }
    for (int a = 0; a < 3; ++a)
      if (hi[a] - lo[a] >= n) return "a plane-wave sphere does not fit the FFT grid";
    int i = 0;
    while (i < npw[k]) {
      int j = i;
      while (j < npw[k] && m[3 * j] == m[3 * i] && m[3 * j + 1] == m[3 * i + 1]) {
        if (j > i && m[3 * j + 2] != m[3 * (j - 1) + 2] + 1) return "a sphere column is not a contiguous run";
        ++j;
      }
      cols[k].push_back(make_int4(m[3 * i], m[3 * i + 1], m[3 * i + 2], j - i));
      starts[k].push_back(i);
      i = j;
    }
    // columns ordered by (m2, m1); rows: runs of columns with equal m2 and consecutive m1,
    // the m2 values consecutive
    const int nc = (int)cols[k].size();
    std::vector<int> perm(nc);
    for (int c = 0; c < nc; ++c) perm[c] = c;
    std::sort(perm.begin(), perm.end(), [&](int x, int y) {
      const int4 a = cols[k][x], b = cols[k][y];
      return a.y < b.y || (a.y == b.y && a.x < b.x);
    });
    std::vector<int4> pc(nc);
    std::vector<int> ps(nc);
    for (int c = 0; c < nc; ++c) { pc[c] = cols[k][perm[c]]; ps[c] = starts[k][perm[c]]; }
    cols[k].swap(pc);
    starts[k].swap(ps);
    int c = 0;
    while (c < nc) {
      int d = c;
      while (d < nc && cols[k][d].y == cols[k][c].y) {
        if (d > c && cols[k][d].x != cols[k][d - 1].x + 1) return "a sphere row is not a contiguous run";
        ++d;
      }
      if (!rows[k].empty() && cols[k][c].y != rows[k].back().x + 1) return "sphere rows are not consecutive";
      rows[k].push_back(make_int4(cols[k][c].y, c, cols[k][c].x, d - c));
      c = d;
    }
    return nullptr;
  };
  const int nth = std::max(1, std::min({(int)std::thread::hardware_concurrency(), 16, nks / 32}));
  if (nth > 1) {
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t)
      pool.emplace_back([&, t] {
        for (int k = t; k < nks; k += nth) kerr[k] = one(k);
      });
    for (auto& th : pool) th.join();
  } else {
    for (int k = 0; k < nks; ++k) kerr[k] = one(k);
  }
  for (int k = 0; k < nks; ++k) {   // the first failing k-point's message, as a serial build gives
    if (kerr[k]) { err = kerr[k]; return false; }
    h.ncol_max = std::max(h.ncol_max, (int)cols[k].size());
    h.nrow_max = std::max(h.nrow_max, (int)rows[k].size());
  }
  h.ncol.resize(nks);
  h.nrow.resize(nks);
  h.col.assign((size_t)nks * h.ncol_max, make_int4(0, 0, 0, 0));
  h.colstart.assign((size_t)nks * h.ncol_max, 0);
  h.row.assign((size_t)nks * h.nrow_max, make_int4(0, 0, 0, 0));
  for (int k = 0; k < nks; ++k) {
    h.ncol[k] = (int)cols[k].size();
    h.nrow[k] = (int)rows[k].size();
    for (int c = 0; c < h.ncol[k]; ++c) {
      h.col[(size_t)k * h.ncol_max + c] = cols[k][c];
      h.colstart[(size_t)k * h.ncol_max + c] = starts[k][c];
    }
    for (int r = 0; r < h.nrow[k]; ++r) h.row[(size_t)k * h.nrow_max + r] = rows[k][r];
  }
  return true;
}

static inline void recip(const double a[3][3], double b[3][3]) {
  const double det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
                     a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  const double f = 2.0 * 3.14159265358979323846 / det;
  // b_i = 2 pi (a_j x a_k) / det
  for (int i = 0; i < 3; ++i) {
    const double* u = a[(i + 1) % 3];
    const double* v = a[(i + 2) % 3];
    b[i][0] = f * (u[1] * v[2] - u[2] * v[1]);
    b[i][1] = f * (u[2] * v[0] - u[0] * v[2]);
    b[i][2] = f * (u[0] * v[1] - u[1] * v[0]);
  }
}

// Orbitals per batch of the per-plane kernel: enough axis-1 lines for the 128 threads when
// orbital-grid planes are staged (their shared memory is the limit), three rounds otherwise
// so that the axis-2 passes (a sphere's rows, ~N/3 lines per orbital) also fill the block.
template <int N, int MODE> struct BO {
  static constexpr int v = (MODE == XY_PASS1_DENS || MODE == XY_PASS2) ? 256 / N : 384 / N;
};

// An FNV-1a-style 64-bit hash over the inputs that determine the u_{vk}(r) grids: the precision, the grid
// side, the k-point and band counts, the spheres of k, the u_k coefficients and the weights
// folded into them (host arrays).
static inline uint64_t ground_state_hash(const ll_system_desc* d) {
  const uint64_t P = 1099511628211ull;
  uint64_t h = 1469598103934665603ull;
  // FNV-1a step over 8-byte words in four interleaved lanes (independent multiply chains),
  // folded into h per array, then the tail words and bytes
  auto feed = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    uint64_t l[4] = {h, h ^ 0x9e3779b97f4a7c15ull, h ^ 0xc2b2ae3d27d4eb4full, h ^ 0x165667b19e3779f9ull};
    size_t i = 0;
    for (; i + 32 <= n; i += 32)
      for (int q = 0; q < 4; ++q) {
        uint64_t wv;
        memcpy(&wv, c + i + 8 * q, 8);
        l[q] = (l[q] ^ wv) * P;
      }
    h = l[0];
    for (int q = 1; q < 4; ++q) h = (h ^ l[q]) * P;
    for (; i + 8 <= n; i += 8) {
      uint64_t wv;
      memcpy(&wv, c + i, 8);
      h = (h ^ wv) * P;
    }
    for (; i < n; ++i) h = (h ^ c[i]) * P;
  };
  feed(&d->precision, sizeof(int));
  feed(&d->nfft, sizeof(int));
  feed(&d->nks, sizeof(int));
  feed(&d->nbnd, sizeof(int));
  long sk = 0;
  for (int k = 0; k < d->nks; ++k) sk += d->npw_k[k];
  feed(d->npw_k, sizeof(int) * (size_t)d->nks);
  feed(d->miller_k, sizeof(int) * 3 * (size_t)sk);
  feed(d->u_k, sizeof(double) * 2 * (size_t)d->nbnd * sk);
  if (d->kweight) feed(d->kweight, sizeof(double) * (size_t)d->nks);   // folded into u_k
  if (d->occ_k) feed(d->occ_k, sizeof(double) * (size_t)d->nks * d->nbnd);   // folded into u_k
  return h;
}

template <typename T>
class Chain : public ChainBase {
 public:
  ~Chain() override {
    for (cudaGraphExec_t& g : graph_)
      if (g) cudaGraphExecDestroy(g);
    for (auto& p : ptrs_) cudaFree(p.first);
  }
  size_t bytes() const override { return bytes_; }

  int create_shared(const ll_system_desc* d, cudaStream_t st, ChainBase* donor, std::string& err) override {
    Chain<T>* dn = dynamic_cast<Chain<T>*>(donor);
    if (!dn) { err = "the sharing chain has another precision"; return LL_EINVAL; }
    if (!dn->ur_share_ || dn->gs_hash_ == 0) { err = "the sharing chain holds no shareable grids"; return LL_EINVAL; }
    donor_ = dn;
    const int rc = create(d, st, err);
    donor_ = nullptr;
    return rc;
  }

  int create(const ll_system_desc* d, cudaStream_t st, std::string& err) override {
    st_ = st;
    N_ = d->nfft;
    nks_ = d->nks;
    nbnd_ = d->nbnd;
    nproj_ = d->nproj;
    approx_ = d->approx;
    flavour_ = d->flavour;
    cap_ = d->max_steps;
    const int n = N_;
    bool ok_n = false;
    for (int s : kGridSides) ok_n |= (s == n);
    if (!ok_n) { err = "unsupported FFT grid side"; return LL_EUNSUPPORTED; }
    if (nks_ < 1 || nbnd_ < 1 || nbnd_ > 32 || nproj_ < 0 || nproj_ > 64 || cap_ < 1) { err = "bad dimensions"; return LL_EINVAL; }
    if (approx_ < 0 || approx_ > 2 || flavour_ < 0 || flavour_ > 1) { err = "bad approx/flavour"; return LL_EINVAL; }
    if (!d->kcart || !d->npw_k || !d->miller_k || !d->npw_kq || !d->miller_kq || !d->u_k || !d->u_kq || !d->eps_k ||
        !d->vloc_r || !d->rho_r || (nproj_ > 0 && (!d->beta_kq || !d->dij))) {
      err = "missing input array";
      return LL_EINVAL;
    }
    if (!build_sphere(nks_, d->npw_k, d->miller_k, n, hk_, err)) return LL_EINVAL;
    if (!build_sphere(nks_, d->npw_kq, d->miller_kq, n, hq_, err)) return LL_EINVAL;
    for (int k = 0; k < nks_; ++k)
      if (d->npw_kq[k] < nbnd_ + 1) { err = "sphere smaller than the occupied manifold"; return LL_EINVAL; }
    {   // the largest |m| of the k+Q spheres on any axis picks the pruning bound of the lines:
        // the tightest built level (tight_prune(N), then N/4) that holds every sphere
      int pmax = 0;
      for (int k = 0; k < nks_; ++k)
        for (int c = 0; c < hq_.ncol[k]; ++c) {
          const int4 cl = hq_.col[(size_t)k * hq_.ncol_max + c];
          pmax = std::max({pmax, std::abs(cl.x), std::abs(cl.y), std::abs(cl.z), std::abs(cl.z + cl.w - 1)});
        }
      const char* pe = getenv("LL_PRUNE");   // 0: unpruned lines; 1: the N/4 level only
      const bool off = pe && pe[0] == '0' && pe[1] == 0, wide = pe && pe[0] == '1' && pe[1] == 0;
      const int tight = tight_prune(n);
      prune_ = off ? 0 : (!wide && tight > 0 && pmax <= tight) ? tight : (pmax <= n / 4 ? n / 4 : 0);
    }
    if (!inputs_finite(d, err, false)) return LL_EINVAL;
    if (d->where != LL_WHERE_HOST && d->where != LL_WHERE_DEVICE) { err = "bad where"; return LL_EINVAL; }
    const bool dev_in = d->where == LL_WHERE_DEVICE;
    // the ground-state hash (host inputs) on another host thread while the device work runs
    std::future<uint64_t> hash_f;
    if (!dev_in) hash_f = std::async(std::launch::async, [d] { return ground_state_hash(d); });
    // k-point weights (stars of the small group of Q) and the group on the grid (Sec. 2.6)
    kscale_.assign(nks_, 1.0);
    if (d->kweight) {
      double sw = 0.0;
      for (int k = 0; k < nks_; ++k) {
        if (!(d->kweight[k] > 0) || !std::isfinite(d->kweight[k])) { err = "k-point weights must be positive"; return LL_EINVAL; }
        sw += d->kweight[k];
      }
      for (int k = 0; k < nks_; ++k) kscale_[k] = std::sqrt(d->kweight[k] * nks_ / sw);
    }
    // a metal (Sec. 2.6): band weights sqrt(f_vk) folded into u_k, the projector and metric tables
    rowscale_.assign((size_t)nks_ * nbnd_, 1.0);
    for (int k = 0; k < nks_; ++k)
      for (int v = 0; v < nbnd_; ++v) rowscale_[(size_t)k * nbnd_ + v] = kscale_[k];
    metal_ = d->occ_k != nullptr;
    if (metal_) {
      if (!d->occ_kq || !d->eps_kq) { err = "a metal needs occ_kq and eps_kq"; return LL_EINVAL; }
      for (long i = 0; i < (long)nks_ * nbnd_; ++i)
        if (!(d->occ_k[i] >= 0.0 && d->occ_k[i] <= 1.0) || !(d->occ_kq[i] >= 0.0 && d->occ_kq[i] <= 1.0)) {
          err = "occupations must lie in [0, 1]";
          return LL_EINVAL;
        }
      const long sz = (long)nks_ * nbnd_ * nbnd_;
      mtab_.assign(4 * sz, 0.0);
      for (int k = 0; k < nks_; ++k)
        for (int m = 0; m < nbnd_; ++m)
          for (int v = 0; v < nbnd_; ++v) {
            const double fv = d->occ_k[(long)k * nbnd_ + v], fm = d->occ_kq[(long)k * nbnd_ + m];
            double c = fv > 0.0 ? std::max(1.0 - fm / fv, 0.0) : 0.0;
            if (c < LL_METAL_CMIN) c = 0.0;
            const double delta = d->eps_kq[(long)k * nbnd_ + m] - d->eps_k[(long)k * nbnd_ + v];
            const long i = ((long)k * nbnd_ + m) * nbnd_ + v;
            const double qh = c > 0.0 ? 1.0 - std::sqrt(c) : 0.0;
            mtab_[i] = c > 0.0 ? qh : 1.0;                        // sp
            mtab_[sz + i] = c > 0.0 ? (1.0 - c) * delta : 0.0;   // da
            mtab_[2 * sz + i] = c > 0.0 ? 0.0 : 1.0;             // keep
            mtab_[3 * sz + i] = qh;                               // qh
          }
      for (int k = 0; k < nks_; ++k)
        for (int v = 0; v < nbnd_; ++v) rowscale_[(size_t)k * nbnd_ + v] *= std::sqrt(d->occ_k[(long)k * nbnd_ + v]);
    }
    if (d->nsym < 0 || (d->nsym > 1 && !d->sym) || d->nsym > 48) { err = "bad symmetry operations"; return LL_EINVAL; }
    nsym_ = d->nsym > 1 ? d->nsym : 1;
    sym_host_.assign(9, 0);
    sym_host_[0] = sym_host_[4] = sym_host_[8] = 1;
    if (d->nsym > 1) {
      sym_host_.assign(d->sym, d->sym + 9 * d->nsym);
      bool has_identity = false;
      for (int i = 0; i < d->nsym; ++i) {
        const int* m = d->sym + 9 * i;
        const long det = (long)m[0] * (m[4] * m[8] - m[5] * m[7]) - (long)m[1] * (m[3] * m[8] - m[5] * m[6]) +
                         (long)m[2] * (m[3] * m[7] - m[4] * m[6]);
        if (det != 1 && det != -1) { err = "a symmetry operation is not unimodular"; return LL_EINVAL; }
        has_identity |= m[0] == 1 && m[4] == 1 && m[8] == 1 && !m[1] && !m[2] && !m[3] && !m[5] && !m[6] && !m[7];
      }
      if (!has_identity) { err = "the symmetry operations lack the identity"; return LL_EINVAL; }
    }
    double b[3][3];
    recip(d->lattice, b);
    omega_ = fabs(d->lattice[0][0] * (d->lattice[1][1] * d->lattice[2][2] - d->lattice[1][2] * d->lattice[2][1]) -
                  d->lattice[0][1] * (d->lattice[1][0] * d->lattice[2][2] - d->lattice[1][2] * d->lattice[2][0]) +
                  d->lattice[0][2] * (d->lattice[1][0] * d->lattice[2][1] - d->lattice[1][1] * d->lattice[2][0]));
    for (int a = 0; a < 3; ++a) q_[a] = d->q_cart[a];
    const long n3 = (long)n * n * n;
    const int pq = hq_.npw_pad, pk = hk_.npw_pad;
    const long vq = (long)nks_ * nbnd_ * pq;  // one batch vector
    nvec_ = (flavour_ == LL_FLAVOUR_NH) ? 2 : 1;

    // Hartree kernel 4 pi / |Q + G|^2 / N^3 over the box, [m3][m2][m1]
    std::vector<T> wh(n3);
    for (int i3 = 0; i3 < n; ++i3)
      for (int i2 = 0; i2 < n; ++i2)
        for (int i1 = 0; i1 < n; ++i1) {
          const int m1 = i1 < n / 2 ? i1 : i1 - n, m2 = i2 < n / 2 ? i2 : i2 - n, m3 = i3 < n / 2 ? i3 : i3 - n;
          double g[3];
          for (int a = 0; a < 3; ++a) g[a] = q_[a] + m1 * b[0][a] + m2 * b[1][a] + m3 * b[2][a];
          const double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
          if (!(g2 > 1e-20)) { err = "Q + G = 0 on the grid (Q is a reciprocal lattice vector)"; return LL_EINVAL; }
          wh[((long)i3 * n + i2) * n + i1] = (T)(4.0 * 3.14159265358979323846 / g2 / (double)n3);
        }
    // kinetic 1/2 |k + Q + G|^2 on sphere(k+Q)
    std::vector<T> kin((size_t)nks_ * pq, T(0));
    for (int k = 0; k < nks_; ++k) {
      const int* m = d->miller_kq + 3L * hq_.off[k];
      for (int i = 0; i < hq_.npw[k]; ++i) {
        double g[3];
        for (int a = 0; a < 3; ++a)
          g[a] = d->kcart[3 * k + a] + q_[a] + m[3 * i] * b[0][a] + m[3 * i + 1] * b[1][a] + m[3 * i + 2] * b[2][a];
        kin[(size_t)k * pq + i] = (T)(0.5 * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
      }
    }
    // The large arrays on the device: the caller's (where = LL_WHERE_DEVICE) or one staging copy
    // of the host arrays; finiteness is checked and the padded tables are built there.
    const long n3l = (long)n * n * n;
    struct Large { const double* p; long len; const char* what; };
    Large large[5] = {{d->u_k, 2L * nbnd_ * hk_.off[nks_], "u_k"},
                      {d->u_kq, 2L * nbnd_ * hq_.off[nks_], "u_kq"},
                      {d->vloc_r, n3l, "vloc_r"},
                      {d->rho_r, n3l, "rho_r"},
                      {d->beta_kq, 2L * nproj_ * hq_.off[nks_], "beta_kq"}};
    double* stage = nullptr;
    {
      int rc0;
      if (!dev_in) {
        long tot = 0;
        for (const Large& a : large) tot += a.len;
        if ((rc0 = alloc(&stage, tot))) return rc0;
        long off = 0;
        for (Large& a : large) {
          if (a.len) LL_CK(cudaMemcpyAsync(stage + off, a.p, a.len * sizeof(double), cudaMemcpyHostToDevice, st_));
          a.p = stage + off;
          off += a.len;
        }
      }
      unsigned long long* first = nullptr;
      if ((rc0 = alloc(&first, 5))) return rc0;
      LL_CK(cudaMemsetAsync(first, 0xFF, 5 * sizeof(unsigned long long), st_));
      for (int i = 0; i < 5; ++i) {
        const Large& a = large[i];
        if (a.len == 0) continue;
        if (dev_in) {
          cudaPointerAttributes at;
          if (cudaPointerGetAttributes(&at, a.p) != cudaSuccess ||
              (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            err = std::string(a.what) + " is not a device pointer (where = LL_WHERE_DEVICE)";
            return LL_EINVAL;
          }
        }
        k_first_nonfinite<<<152, 256, 0, st_>>>(a.p, a.len, first + i);
      }
      unsigned long long h[5];
      LL_CK(cudaMemcpyAsync(h, first, sizeof(h), cudaMemcpyDeviceToHost, st_));
      LL_CK(cudaStreamSynchronize(st_));
      for (int i = 0; i < 5; ++i)
        if (large[i].len && h[i] != ~0ull) {
          err = std::string("non-finite value in ") + large[i].what + " at index " + std::to_string(h[i]);
          return LL_EINVAL;
        }
      release(first);
    }
    gs_hash_ = dev_in ? 0 : hash_f.get();
    if (donor_) {
      if (dev_in) { err = "grids are shared between chains of host inputs only"; return LL_EINVAL; }
      if (gs_hash_ != donor_->gs_hash_ || donor_->N_ != N_ || donor_->nks_ != nks_ || donor_->nbnd_ != nbnd_) {
        err = "the ground state differs from the sharing chain's (grid, k-points, bands, sphere(k) or u_k)";
        return LL_EINVAL;
      }
    }
    // padded orbital tables and grids transposed to [j3][j2][j1]: built on the device from the
    // large arrays (the caller's device arrays or their staging copy) by k_pad_rows / k_grids_in
    const long bkq_len = nproj_ ? (long)nks_ * nproj_ * pq : 1;

    int rc;
    if ((rc = tw_tables_upload(st_)) != cudaSuccess) { err = "twiddle upload failed"; return LL_ECUDA; }
    // device buffers
    if ((rc = upload_sphere(hk_, dk_, err)) || (rc = upload_sphere(hq_, dq_, err))) return rc;
    cb_ncol_ = round_up(std::max(hk_.ncol_max, hq_.ncol_max), 2);   // even: 16-byte rows in FP32
    const int norb = nvec_ * nks_ * nbnd_;
    {
      int dev = 0, sms = 0;
      if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        nsm_ = sms;
      cudaGetLastError();
    }
    ngroups_ = groups_for(norb);
    // per-k work: fused (one CTA holds a k block) when it fits in shared memory, else split
    // over chunks of plane waves (LL_SPLIT_PERK=1 in the environment forces the split path)
    {
      // one CTA per (k, group of bpc bands): the largest band group whose two vectors, dot
      // coefficients, scratch and static arrays fit one CTA's shared memory (all bands of a
      // k-point when they fit: the Lanczos partials are then one per k)
      auto fused = [&](int b) {
        bpc_ = b;
        return 2 * (size_t)b * pq * sizeof(cplx<T>) + (size_t)std::max(nproj_, nbnd_) * b * sizeof(cplx<double>) +
               red_bytes(256) + 32 * 32 * sizeof(cplx<T>) + 4096;
      };
      int best = 0;
      for (int b = nbnd_; b >= 1 && !best; --b)
        if (nbnd_ % b == 0 && fused(b) <= 227 * 1024) best = b;
      bpc_ = best > 0 ? best : nbnd_;
      ngrp_ = nbnd_ / bpc_;
      const char* env = getenv("LL_SPLIT_PERK");
      // the chunked path also where the band groups are small: per-group CTAs would read the
      // projectors and U_{k+Q} once per group (32 times per k on the 16-atom cell)
      split_ = best == 0 || 4 * best < nbnd_ || (env && env[0] == '1' && env[1] == 0);
      nchunk_ = split_ ? (pq + kChunk - 1) / kChunk : 1;
      npk_ = split_ ? nchunk_ : ngrp_;
      // FP32 path: the split path's dot blocks on the tensor cores (tcproj.cuh) where their
      // rows fit one M = 128 tile (LL_TC=0 in the environment keeps them on the CUDA cores)
      const char* tce = getenv("LL_TC");
      const bool tc = std::is_same<T, float>::value && split_ && !(tce && tce[0] == '0' && tce[1] == 0);
      tc_nb_op_ = round_up(3 * nbnd_, 32);
      tc_nb_u_ = round_up(nbnd_, 32);
      tc_op_ = tc && nproj_ + 2 * nbnd_ <= 128 && tc_nb_op_ <= 256 && nproj_ + 3 * nbnd_ <= kTcMaxRows;
      tc_u_ = tc && 2 * nbnd_ <= 128;
      tc_u2_ = tc && 4 * nbnd_ <= 128;
      tc_nb_ap_ = round_up(2 * nbnd_, 32);
      tc_ap_ = tc && tc_nb_ap_ <= 128;
    }
    const long nzp = (long)nks_ * npk_;               // partials per vector and step
    const long nzv = nzp * nvec_;
    if ((rc = alloc(&whart_, n3)) || (rc = alloc(&kin_, (long)nks_ * pq)) || (rc = alloc(&uk_, (long)nks_ * nbnd_ * pk)) ||
        (rc = alloc(&ukq_, vq)) || (rc = alloc(&bkq_, bkq_len)) || (rc = alloc(&eps_, (long)nks_ * nbnd_)) ||
        (rc = alloc(&dij_, std::max(1, nproj_))) || (rc = alloc(&vloc_, n3)) || (rc = alloc(&rho_, n3)) ||
        (rc = alloc(&fxc_, n3)) || (rc = ur_alloc((long)nks_ * nbnd_ * n3)) ||
        (rc = alloc(&cbuf_, (long)norb * n * cb_ncol_)) || (rc = alloc(&nprt_, (long)ngroups_ * n3)) ||
        (rc = alloc(&nr_, n3)) || (rc = alloc(&ng_, n3)) || (rc = alloc(&vpr_, n3)) ||
        (rc = alloc(&y_, vq)) || (rc = alloc(&map_, (long)nks_ * pq)) || (rc = alloc(&part_, std::max(2L * nks_, nzv))) ||
        (rc = alloc(&spart_, nzp)) || (rc = alloc(&vecs_, 3L * nvec_ * vq)) ||
        (rc = alloc(&beta_, cap_ + 2)) || (rc = alloc(&gamma_, cap_ + 2)) || (rc = alloc(&z_, cap_ + 1)) ||
        (rc = alloc(&zpart_, (long)(cap_ + 1) * nzp)) || (rc = alloc(&err_, 2)) || (rc = alloc(&jdev_, 1)))
      return rc;
    if (metal_) {
      const long sz = (long)nks_ * nbnd_ * nbnd_;
      if ((rc = alloc(&mc_, 4 * sz)) || (rc = alloc(&img_, nvec_ * vq)) || (rc = alloc(&zp_, nvec_ * sz)) ||
          (rc = alloc(&mcorr_, (long)nvec_ * nks_)))
        return rc;
      LL_CK(cudaMemcpyAsync(mc_, mtab_.data(), 4 * sz * sizeof(double), cudaMemcpyHostToDevice, st_));
      md_ = MetalDev{mc_, mc_ + sz, mc_ + 2 * sz, mc_ + 3 * sz};
    }
    {
      const char* g = getenv("LL_GRAPHS");
      use_graphs_ = use_graphs_ && !(g && g[0] == '0' && g[1] == 0);
      const char* xp = getenv("LL_XY_PAIR");   // 1: lane pairs for every even N, 0: never (k_xy)
      xy_pair_ = (xp && xp[1] == 0 && (xp[0] == '0' || xp[0] == '1')) ? xp[0] - '0' : -1;
    }
    // chunk partials: U^H x per vector (two per vector on the non-Hermitian update), B^H x
    if (split_ && ((rc = alloc(&sp_s_, 2 * nzv * nbnd_ * nbnd_)) || (rc = alloc(&sp_c_, nzv * std::max(1, nproj_ * nbnd_))) ||
                   (rc = alloc(&ub_, (long)nks_ * nbnd_ * std::max(1, nproj_))) ||
                   (rc = alloc(&sp_coef_, nvec_ * (long)nks_ * (nproj_ + nbnd_) * nbnd_))))
      return rc;
    (void)err;
    LL_CK(cudaMemcpyAsync(whart_, wh.data(), n3 * sizeof(T), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(kin_, kin.data(), kin.size() * sizeof(T), cudaMemcpyHostToDevice, st_));
    {
      int *offk = nullptr, *offq = nullptr;
      double* ksc = nullptr;
      if ((rc = alloc(&offk, nks_ + 1)) || (rc = alloc(&offq, nks_ + 1)) || (rc = alloc(&ksc, (long)nks_ * nbnd_))) return rc;
      LL_CK(cudaMemcpyAsync(offk, hk_.off.data(), (nks_ + 1) * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(offq, hq_.off.data(), (nks_ + 1) * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(ksc, rowscale_.data(), (size_t)nks_ * nbnd_ * sizeof(double), cudaMemcpyHostToDevice, st_));
      k_pad_rows<T><<<dim3(nks_, nbnd_), 256, 0, st_>>>(large[0].p, offk, dk_.npw, nbnd_, hk_.npw_pad, ksc, uk_);
      k_pad_rows<T><<<dim3(nks_, nbnd_), 256, 0, st_>>>(large[1].p, offq, dq_.npw, nbnd_, pq, nullptr, ukq_);
      if (nproj_) k_pad_rows<T><<<dim3(nks_, nproj_), 256, 0, st_>>>(large[4].p, offq, dq_.npw, nproj_, pq, nullptr, bkq_);
      k_grids_in<T><<<256, 256, 0, st_>>>(n, large[2].p, large[3].p, vloc_, rho_);
      LL_CK(cudaGetLastError());
      LL_CK(cudaStreamSynchronize(st_));   // the caller may reuse its arrays once ll_create returns
      release(offk);
      release(offq);
      release(ksc);
      release(stage);
    }
    LL_CK(cudaMemcpyAsync(eps_, d->eps_k, sizeof(double) * nks_ * nbnd_, cudaMemcpyHostToDevice, st_));
    if (nproj_) LL_CK(cudaMemcpyAsync(dij_, d->dij, sizeof(double) * nproj_, cudaMemcpyHostToDevice, st_));
    if (nsym_ > 1) {
      if ((rc = alloc(&sym_, 9L * nsym_))) return rc;
      LL_CK(cudaMemcpyAsync(sym_, sym_host_.data(), 9L * nsym_ * sizeof(int), cudaMemcpyHostToDevice, st_));
    }
    LL_CK(cudaMemsetAsync(err_, 0, 2 * sizeof(int), st_));
    LL_CK(cudaMemsetAsync(vecs_, 0, 3L * nvec_ * vq * sizeof(cplx<T>), st_));
    LL_CK(cudaMemsetAsync(zpart_, 0, (long)(cap_ + 1) * nzp * sizeof(cplx<double>), st_));
    k_fxc<T><<<256, 256, 0, st_>>>(n3, rho_, fxc_, approx_ == LL_APPROX_TDDFT ? 1 : 0);
    LL_CK(cudaGetLastError());
    if (split_ && nproj_ > 0) {  // U^H B per k (the KB part of P_c on the split path)
      const size_t sm = (size_t)(nbnd_ + nproj_) * kTileP * sizeof(cplx<T>);
      if ((rc = set_smem(k_sp_ub<T>, sm, err))) return rc;
      k_sp_ub<T><<<dim3(nks_, nchunk_), 256, sm, st_>>>(nbnd_, pq, dq_.npw, nchunk_, nproj_, ukq_, bkq_, sp_c_);
      k_sp_reduce<<<nks_, 256, 0, st_>>>(nchunk_, nbnd_ * nproj_, sp_c_, ub_);
      LL_CK(cudaGetLastError());
    }

    // index map sphere(k+Q) -> sphere(k) (on the device, from the Miller lists)
    {
      int *mk = nullptr, *mq = nullptr, *ok = nullptr, *oq = nullptr, *nk = nullptr, *nq = nullptr;
      if ((rc = alloc(&mk, 3L * hk_.off[nks_])) || (rc = alloc(&mq, 3L * hq_.off[nks_])) || (rc = alloc(&ok, nks_ + 1)) ||
          (rc = alloc(&oq, nks_ + 1)) || (rc = alloc(&nk, nks_)) || (rc = alloc(&nq, nks_)))
        return rc;
      LL_CK(cudaMemcpyAsync(mk, d->miller_k, 3L * hk_.off[nks_] * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(mq, d->miller_kq, 3L * hq_.off[nks_] * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(ok, hk_.off.data(), (nks_ + 1) * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(oq, hq_.off.data(), (nks_ + 1) * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(nk, d->npw_k, nks_ * sizeof(int), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(nq, d->npw_kq, nks_ * sizeof(int), cudaMemcpyHostToDevice, st_));
      k_intersection_map<<<nks_, 128, 0, st_>>>(nks_, ok, nk, mk, oq, nq, mq, pq, map_);
      LL_CK(cudaGetLastError());
      LL_CK(cudaStreamSynchronize(st_));
      for (int* p : {mk, mq, ok, oq, nk, nq}) release(p);
    }
    // y = P_c (u_k on sphere(k+Q))   (Eq. 28).  A metal: Q^-1 of the start P_{c,v} u_k (u_k with
    // sqrt(f_v) folded in), i.e. Q P'_v u_k
    k_gather_y<T><<<dim3(nks_, nbnd_), 128, 0, st_>>>(nks_, nbnd_, pq, pk, map_, uk_, y_);
    k_project<T><<<dim3(nks_, 1, nbnd_), 128, 0, st_>>>(nks_, nbnd_, pq, dq_.npw, ukq_, y_, md_.keep);
    if (metal_) k_project<T><<<dim3(nks_, 1, nbnd_), 128, 0, st_>>>(nks_, nbnd_, pq, dq_.npw, ukq_, y_, md_.qh);
    LL_CK(cudaGetLastError());
    // u_{vk}(r) grids: columns of sphere(k), then the planes (unless a chain of the same ground
    // state lends its grids)
    if (!donor_) {
      if ((rc = launch_zinv(dk_, uk_, 1)) || (rc = launch_xy(dk_, nks_ * nbnd_, 0, -1, 2, err))) return rc;
      LL_CK(cudaGetLastError());
    }


    // the plane pass's kernel variant and batch per mode, timed on this system (cached per shape)
    if ((rc = tune_plane_pass(err))) return rc;

    // start of the recursion
    if (flavour_ == LL_FLAVOUR_PH) {
      LL_CK(cudaMemcpyAsync(R(), y_, vq * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st_));
      if ((rc = op(1, R(), X(), -1, err))) return rc;               // X_1 = D y
      std::vector<double> hp(nzp);
      LL_CK(cudaMemcpyAsync(hp.data(), part_, nzp * sizeof(double), cudaMemcpyDeviceToHost, st_));
      LL_CK(cudaStreamSynchronize(st_));
      double s = 0;
      for (double v : hp) s += v;
      s /= nks_;
      if (!(s > 0)) { err = "D is not positive on the starting vector"; return LL_ENOTPD; }
      tol_ = 1e-28 * s;
    } else {
      k_dot_re<T><<<nks_, 128, 0, st_>>>(nks_, nbnd_, pq, y_, y_, part_);
      std::vector<double> hp(nks_);
      LL_CK(cudaMemcpyAsync(hp.data(), part_, nks_ * sizeof(double), cudaMemcpyDeviceToHost, st_));
      LL_CK(cudaStreamSynchronize(st_));
      double s = 0;
      for (double v : hp) s += v;
      s /= nks_;
      if (!(s > 0)) { err = "the starting vector vanishes"; return LL_EINVAL; }
      const double b1 = sqrt(s);
      tol_ = 1e-28 * s;
      k_scale<T><<<256, 256, 0, st_>>>(vq, y_, 1.0 / b1, Vc());
      k_scale<T><<<256, 256, 0, st_>>>(vq, y_, 1.0 / b1, Wc());
      cplx<double> g1 = mk(b1, 0.0);
      LL_CK(cudaMemcpyAsync(beta_, &b1, sizeof(double), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaMemcpyAsync(gamma_, &g1, sizeof(g1), cudaMemcpyHostToDevice, st_));
      LL_CK(cudaGetLastError());
    }
    LL_CK(cudaStreamSynchronize(st_));
    steps_ = 0;
    queued_ = 0;
    return oob_check(err);
  }

  int lanczos(int n, double* beta, double* gamma, double* z, int* done, std::string& err) override {
    int rc = enqueue(n, err);
    if (rc != LL_OK) {
      if (done) *done = steps_;
      return rc;
    }
    return collect(beta, gamma, z, done, err);
  }

  int steps_queued() const override { return queued_; }

  int enqueue(int n, std::string& err) override {
    if (n < 0 || queued_ + n > cap_) { err = "more steps than max_steps"; return LL_EINVAL; }
    if (stopped_) { err = "the chain stopped at a breakdown"; return LL_EBREAKDOWN; }
    int rc;
    const int pq = hq_.npw_pad;
    const size_t smem_nh = 2 * (size_t)bpc_ * pq * sizeof(cplx<T>) + (size_t)nbnd_ * bpc_ * sizeof(cplx<double>) +
                           16 * 4 * sizeof(double);
    Coef co{beta_, gamma_, zpart_, err_};
    if (flavour_ == LL_FLAVOUR_PH && n > 0) {
      k_step_set<<<1, 1, 0, st_>>>(jdev_, queued_ + 1);
      LL_CK(cudaGetLastError());
      prof_.count(LL_PROF_UPDATE);
    }
    for (int s = 0; s < n; ++s) {
      const int j = queued_ + s + 1;
      if (flavour_ == LL_FLAVOUR_PH) {
        const int par = j % 2;
        // a step of each parity is captured into a CUDA graph once one has run eagerly (every
        // lazily set kernel attribute and launch shape is then fixed) and replayed after that;
        // not while profiling, and not on the legacy default stream, which cannot be captured
        if (use_graphs_ && !prof_.on && st_ != nullptr && eager_done_[par] && !graph_[par]) {
          if ((rc = capture_step(j, err))) return rc;
        }
        if (graph_[par] && !prof_.on) {
          LL_CK(cudaGraphLaunch(graph_[par], st_));
          count_step(j);
        } else {
          if ((rc = ph_step(j, err))) return rc;
          eager_done_[par] = true;
        }
      } else {
        const int upper = (j % 2 == 0) ? 1 : 0;
        // L v_j: D + K on an upper v; L^dag w_j: D + K on a lower w
        const int dens = (approx_ == LL_APPROX_IPA) ? -1 : (upper ? 0 : 1);
        if ((rc = op(2, Vc(), XV(), dens, err))) return rc;
        const int u0 = prof_.mark(st_);
        if (split_) {  // the update split over plane-wave chunks (split.cuh)
          const size_t sm = (size_t)(2 * nbnd_) * kTileP * sizeof(cplx<T>);
          if ((rc = set_smem(k_sp_nh_start<T>, sm, err))) return rc;
          k_sp_nh_start<T><<<dim3(nks_, nchunk_), 256, sm, st_>>>(j, upper, nks_, nbnd_, pq, dq_.npw, nchunk_, XV(),
                                                                  XW(), VpNH(), Wp(), Vc(), y_, ukq_, co, sp_s_,
                                                                  tc_u2_ ? 0 : 1);
          if (tc_u2_ && (rc = tc_dots<TC_U2>(1, tc_nb_u_, nullptr, XV(), XW(), nullptr, sp_s_, err))) return rc;
          k_sp_nh_proj<T><<<dim3(nks_, nchunk_), 256, 0, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, XV(), XW(), ukq_,
                                                                sp_s_, spart_, md_.keep);
          prof_.count(LL_PROF_UPDATE, 1);
        } else {
          if ((rc = set_smem(k_nh_update<T>, smem_nh, err))) return rc;
          k_nh_update<T><<<dim3(nks_, ngrp_), 128, smem_nh, st_>>>(j, upper, nks_, nbnd_, bpc_, pq, dq_.npw, XV(),
                                                                   XW(), VpNH(), Wp(),
                                                      Vc(), y_, ukq_, co, spart_, md_.keep);
        }
        k_nh_normalize<T><<<nks_, 128, 0, st_>>>(j, nks_, nbnd_, pq, npk_, spart_, XV(), XW(), Vc(), VpNH(), Wc(),
                                                 Wp(), co, tol_);
        prof_.count(LL_PROF_UPDATE, 2);
        prof_.span(LL_PROF_UPDATE, u0, prof_.mark(st_));
      }
      LL_CK(cudaGetLastError());
    }
    if (n > 0) {
      k_reduce_z<<<(n + 127) / 128, 128, 0, st_>>>(zpart_, nks_ * npk_, nks_, queued_, queued_ + n, z_);
      LL_CK(cudaGetLastError());
      prof_.count(LL_PROF_UPDATE);
    }
    queued_ += n;
    return LL_OK;
  }

  // One pseudo-Hermitian step (the step index comes from the device counter jdev_, which the
  // step advances at its end): update of the Lanczos vectors and the axis-3 inverse FFT of
  // r_{j+1}, then the rest of the operator (D + K when j is odd: r_{j+1} is then upper).
  int ph_step(int j, std::string& err) {
    int rc;
    const int u0 = prof_.mark(st_);
    if ((rc = launch_zinv_ph(j, err))) return rc;
    prof_.span(LL_PROF_ZINV, u0, prof_.mark(st_));
    const int dens = (j % 2 == 1 && approx_ != LL_APPROX_IPA) ? 0 : -1;
    if ((rc = op_rest(1, R(), X(), dens, err))) return rc;
    k_step_next<<<1, 1, 0, st_>>>(jdev_);
    prof_.count(LL_PROF_ZINV, split_ ? 4 : 2);
    prof_.count(LL_PROF_UPDATE);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  // launch counts of a replayed step (the same kernels as ph_step)
  void count_step(int j) {
    prof_.count(LL_PROF_ZINV, (split_ ? 4 : 2) + (metal_ ? (split_ ? 3 : 1) : 0));
    prof_.count(LL_PROF_UPDATE);
    prof_.count(LL_PROF_XY1);
    if (j % 2 == 1 && approx_ != LL_APPROX_IPA) {
      prof_.count(LL_PROF_HXC, 3);
      prof_.count(LL_PROF_XY2);
    }
    prof_.count(LL_PROF_ZFWD, split_ ? 4 + (metal_ ? 1 : 0) : 1);
  }
  int capture_step(int j, std::string& err) {
    cudaGraph_t g = nullptr;
    LL_CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    // the captured launches are counted when the graph is replayed, not here (profiling is
    // off during a capture, so only the launch counters move)
    long long saved[LL_NPROF], saved_total = prof_.total;
    for (int c = 0; c < LL_NPROF; ++c) saved[c] = prof_.launches[c];
    int rc = ph_step(j, err);
    for (int c = 0; c < LL_NPROF; ++c) prof_.launches[c] = saved[c];
    prof_.total = saved_total;
    cudaError_t e = cudaStreamEndCapture(st_, &g);
    if (rc != LL_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) { err = std::string("step capture: ") + cudaGetErrorString(e); return LL_ECUDA; }
    e = cudaGraphInstantiate(&graph_[j % 2], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      graph_[j % 2] = nullptr;
      err = std::string("step graph: ") + cudaGetErrorString(e);
      return LL_ECUDA;
    }
    return LL_OK;
  }

  // The bounds-checked build (-DLL_CHECK): LL_EINVAL when a kernel met an index outside its
  // table's range since the library was loaded; the plain build: always LL_OK.
  int oob_check(std::string& err) {
#ifdef LL_CHECK
    int line = 0;
    LL_CK(cudaMemcpyFromSymbolAsync(&line, g_oob_line, sizeof(int), 0, cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    if (line) {
      err = "index out of bounds in a kernel (kernel source line " + std::to_string(line) + ")";
      return LL_EINVAL;
    }
#endif
    (void)err;
    return LL_OK;
  }

  int collect(double* beta, double* gamma, double* z, int* done, std::string& err) override {
    if (int rc = oob_check(err)) return rc;
    int herr[2];
    LL_CK(cudaMemcpyAsync(herr, err_, sizeof(herr), cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    steps_ = queued_;
    int status = LL_OK;
    if (herr[0] != DEV_OK && herr[0] != DEV_TIMEOUT && herr[1] - 1 >= queued_) {
      // the breakdown is that of the coefficient after the last one asked for (the
      // non-Hermitian step forms beta_{j+1} with z_j): every coefficient asked for is valid;
      // the chain stops, and the next call reports it
      stopped_ = true;
    } else if (herr[0] != DEV_OK) {
      steps_ = std::min(steps_, herr[1] - 1);
      queued_ = steps_;
      status = (herr[0] == DEV_NOTPD) ? LL_ENOTPD : (herr[0] == DEV_TIMEOUT ? LL_ETIMEOUT : LL_EBREAKDOWN);
      err = (status == LL_ENOTPD)     ? "pseudo-Hermitian metric not positive"
            : (status == LL_ETIMEOUT) ? "a bounded tensor-core wait gave up"
                                      : "Lanczos breakdown";
      stopped_ = true;
    }
    if (done) *done = steps_;
    if (steps_ > 0) {
      if (beta) LL_CK(cudaMemcpyAsync(beta, beta_, steps_ * sizeof(double), cudaMemcpyDeviceToHost, st_));
      if (gamma) LL_CK(cudaMemcpyAsync(gamma, gamma_, steps_ * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st_));
      if (z) LL_CK(cudaMemcpyAsync(z, z_, steps_ * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st_));
      LL_CK(cudaStreamSynchronize(st_));
    }
    return status;
  }

  int steps() const override { return steps_; }
  void set_graphs(bool on) override { use_graphs_ = use_graphs_ && on; }

  int spectrum(int m, int kind, int m_total, const double* w_ev, int nw, double eta_ev, double* chi, double* ei,
               double* e, std::string& err) override {
    if (m <= 0 || m > steps_) m = steps_;
    if (kind == LL_EXTRAP_NO || m_total < m) m_total = m;
    if (m < 1 || nw < 1) { err = "no coefficients or no frequencies"; return LL_EINVAL; }
    int rc;
    if (nw > spec_cap_) {
      release(spec_w_); release(spec_out_);
      spec_w_ = nullptr; spec_out_ = nullptr;
      if ((rc = alloc(&spec_w_, nw)) || (rc = alloc(&spec_out_, 3L * nw))) return rc;
      spec_cap_ = nw;
    }
    const double ha = 27.211386245988;
    std::vector<double> w(nw);
    for (int i = 0; i < nw; ++i) w[i] = w_ev[i] / ha;
    LL_CK(cudaMemcpyAsync(spec_w_, w.data(), nw * sizeof(double), cudaMemcpyHostToDevice, st_));
    const double q2 = q_[0] * q_[0] + q_[1] * q_[1] + q_[2] * q_[2];
    if (m_total > m) {
      if (!tail_ && (rc = alloc(&tail_, 1))) return rc;
      k_extrap_tail<<<1, 256, 0, st_>>>(m, kind, beta_, gamma_, tail_);
    }
    k_spectrum<<<(nw + 127) / 128, 128, 0, st_>>>(m, m_total, m_total > m ? tail_ : nullptr, beta_, gamma_, z_, nw,
                                                  spec_w_, eta_ev / ha, 4.0 / omega_,
                                                  4.0 * 3.14159265358979323846 / q2, spec_out_, spec_out_ + nw,
                                                  spec_out_ + 2L * nw);
    LL_CK(cudaGetLastError());
    if (chi) LL_CK(cudaMemcpyAsync(chi, spec_out_, nw * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st_));
    if (ei) LL_CK(cudaMemcpyAsync(ei, spec_out_ + nw, nw * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st_));
    if (e) LL_CK(cudaMemcpyAsync(e, spec_out_ + 2L * nw, nw * sizeof(cplx<double>), cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    return LL_OK;
  }

  int apply(int upper, const double* x, double* out, std::string& err) override {
    int rc;
    const long vq = (long)nks_ * nbnd_ * hq_.npw_pad;
    if (!scratch_ && (rc = alloc(&scratch_, 2 * vq))) return rc;
    std::vector<cplx<T>> h = pad_batch(x, hq_, nbnd_);
    LL_CK(cudaMemcpyAsync(scratch_, h.data(), vq * sizeof(cplx<T>), cudaMemcpyHostToDevice, st_));
    // a one-vector application reuses the cbuf/tbuf sized for nvec_ >= 1
    if ((rc = op(1, scratch_, scratch_ + vq, (upper && approx_ != LL_APPROX_IPA) ? 0 : -1, err))) return rc;
    LL_CK(cudaMemcpyAsync(h.data(), scratch_ + vq, vq * sizeof(cplx<T>), cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    if ((rc = oob_check(err))) return rc;
    unpad_batch(h, hq_, nbnd_, out);
    return LL_OK;
  }

  int get_map(int* out, std::string& err) override {
    std::vector<int> h((size_t)nks_ * hq_.npw_pad);
    LL_CK(cudaMemcpyAsync(h.data(), map_, h.size() * sizeof(int), cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    for (int k = 0; k < nks_; ++k)
      memcpy(out + hq_.off[k], h.data() + (size_t)k * hq_.npw_pad, hq_.npw[k] * sizeof(int));
    return LL_OK;
  }

  int get_start(double* y, std::string& err) override {
    std::vector<cplx<T>> h((size_t)nks_ * nbnd_ * hq_.npw_pad);
    LL_CK(cudaMemcpyAsync(h.data(), y_, h.size() * sizeof(cplx<T>), cudaMemcpyDeviceToHost, st_));
    LL_CK(cudaStreamSynchronize(st_));
    unpad_batch(h, hq_, nbnd_, y);
    return LL_OK;
  }

  int profile(int enable, std::string& err) override {
    LL_CK(cudaStreamSynchronize(st_));
    if (enable) prof_.reset();
    prof_.on = enable != 0;
    return LL_OK;
  }

  int profile_read(double* ms, long long* launches, long long* total, std::string& err) override {
    LL_CK(cudaStreamSynchronize(st_));
    for (int c = 0; c < LL_NPROF; ++c) {
      if (ms) ms[c] = 0.0;
      if (launches) launches[c] = prof_.launches[c];
    }
    if (total) *total = prof_.total;
    if (ms)
      for (size_t i = 0; i < prof_.cls.size(); ++i) {
        float t = 0.f;
        LL_CK(cudaEventElapsedTime(&t, prof_.pool[prof_.ea[i]], prof_.pool[prof_.eb[i]]));
        ms[prof_.cls[i]] += t;
      }
    return LL_OK;
  }

 private:
  // one batch operator application on nvec contiguous vectors (Eqs. 24-28)
  int op(int nvec, const cplx<T>* in, cplx<T>* out, int dens_vec, std::string& err) {
    int rc;
    const int e0 = prof_.mark(st_);
    const cplx<T>* zin = metal_image(in, nvec);
    if (!zin) { err = "metal image launch"; return LL_ECUDA; }
    if ((rc = launch_zinv(dq_, zin, nvec))) { err = "zinv launch"; return rc; }
    prof_.count(LL_PROF_ZINV);
    prof_.span(LL_PROF_ZINV, e0, prof_.mark(st_));
    return op_rest(nvec, in, out, dens_vec, err);
  }

  // A metal: the image Q z of the batch vectors at `in` (and Z = U^H z) that the FFT pipeline
  // reads in their place; an insulator: `in` itself.
  const cplx<T>* metal_image(const cplx<T>* in, int nvec) {
    if (!metal_) return in;
    if (split_) {   // over plane-wave chunks: U^H z, the coefficients qh Z, img = z - U (qh Z)
      const int pq = hq_.npw_pad;
      const long vq = (long)nks_ * nbnd_ * pq;
      cudaMemcpyAsync(img_, in, nvec * vq * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st_);
      const size_t sm_d = (size_t)(2 * nbnd_) * kTileP * sizeof(cplx<T>);
      const size_t sm_a = (size_t)nbnd_ * (nbnd_ + kSub) * sizeof(cplx<T>);
      std::string e;
      if (set_smem(k_sp_dots<T>, sm_d, e) || set_smem(k_sp_apply<T>, sm_a, e)) return nullptr;
      k_sp_dots<T><<<dim3(nks_, nvec, nchunk_), 256, sm_d, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, 0, in, in, ukq_,
                                                                  bkq_, sp_c_, sp_s_);
      k_sp_coef<T><<<nks_ * nvec, 256, 0, st_>>>(nks_, nbnd_, nchunk_, 0, dij_, ub_, sp_c_, sp_s_, sp_coef_, 3, md_,
                                                 zp_, nullptr);
      k_sp_apply<T><<<dim3(nks_, nvec, nchunk_), 256, sm_a, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, 0, nullptr,
                                                                   img_, ukq_, bkq_, sp_coef_, nullptr);
      prof_.count(LL_PROF_ZINV, 3);
      return img_;
    }
    k_metal_image<T><<<dim3(nks_, nvec), 128, 0, st_>>>(nks_, nbnd_, hq_.npw_pad, dq_.npw, ukq_, in, img_, zp_, md_);
    prof_.count(LL_PROF_ZINV);
    return img_;
  }

  // everything after the axis-3 inverse FFT: planes, response potential, axis-3 forward FFT
  // fused with the per-k projections
  int op_rest(int nvec, const cplx<T>* in, cplx<T>* out, int dens_vec, std::string& err) {
    int rc;
    const int e1 = prof_.mark(st_);
    if ((rc = launch_xy(dq_, nvec * nks_ * nbnd_, 0, dens_vec, 0, err))) return rc;
    prof_.count(LL_PROF_XY1);
    int e2 = prof_.mark(st_);
    prof_.span(LL_PROF_XY1, e1, e2);
    if (dens_vec >= 0) {
      if ((rc = launch_hxc(err))) return rc;
      prof_.count(LL_PROF_HXC, 3);
      const int e3 = prof_.mark(st_);
      prof_.span(LL_PROF_HXC, e2, e3);
      if ((rc = launch_xy(dq_, nks_ * nbnd_, dens_vec * nks_ * nbnd_, dens_vec, 1, err))) return rc;
      prof_.count(LL_PROF_XY2);
      e2 = prof_.mark(st_);
      prof_.span(LL_PROF_XY2, e3, e2);
    }
    if ((rc = launch_zfwd_proj(nvec, in, out, err))) return rc;
    prof_.count(LL_PROF_ZFWD, split_ ? 4 + (metal_ ? 1 : 0) : 1);
    prof_.span(LL_PROF_ZFWD, e2, prof_.mark(st_));
    return LL_OK;
  }

  // reduction scratch of the per-k dot routines: max(16, 2*ni*nj) doubles per warp
  size_t red_bytes(int threads) const {
    const int pairs = std::max(std::max(nproj_, nbnd_) * std::max(bpc_, 1), 8);
    return (size_t)(threads / 32) * 2 * pairs * sizeof(double);
  }
  template <int N>
  int zfwd_proj_n(int nvec, const cplx<T>* in, cplx<T>* out, std::string& err) {
    if (split_) return zfwd_split_n<N>(nvec, in, out, err);
    const size_t smem = 2 * (size_t)bpc_ * hq_.npw_pad * sizeof(cplx<T>) +
                        (size_t)std::max(nproj_, nbnd_) * bpc_ * sizeof(cplx<double>) + red_bytes(256);
    int rc;
    auto kern = k_zfwd_proj<T, N>;
    if constexpr (tight_prune(N) > 0)
      if (prune_ == tight_prune(N)) kern = k_zfwd_proj<T, N, tight_prune(N)>;
    if (prune_ == N / 4) kern = k_zfwd_proj<T, N, N / 4>;
    if ((rc = set_smem(kern, smem, err))) return rc;
    kern<<<dim3(nks_, nvec, ngrp_), 256, smem, st_>>>(dq_, nbnd_, bpc_, cbuf_, cb_ncol_,
                                                                    metal_ ? img_ : in, kin_, eps_, ukq_, bkq_,
                                                                    dij_, nproj_, out, part_, md_, zp_);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  int launch_zfwd_proj(int nvec, const cplx<T>* in, cplx<T>* out, std::string& err) {
    switch (N_) {
      case 12: return zfwd_proj_n<12>(nvec, in, out, err);
      case 16: return zfwd_proj_n<16>(nvec, in, out, err);
      case 18: return zfwd_proj_n<18>(nvec, in, out, err);
      case 24: return zfwd_proj_n<24>(nvec, in, out, err);
      case 32: return zfwd_proj_n<32>(nvec, in, out, err);
      case 36: return zfwd_proj_n<36>(nvec, in, out, err);
      case 48: return zfwd_proj_n<48>(nvec, in, out, err);
    }
    return LL_EUNSUPPORTED;
  }
  // The split path's chunk dot blocks on the tensor cores (FP32 path only; tcproj.cuh).
  template <int MODE>
  int tc_dots(int nvec, int nb, const cplx<T>* x, const cplx<T>* t, const cplx<T>* t2, cplx<double>* cpart,
              cplx<double>* spart, std::string& err) {
    if constexpr (std::is_same<T, float>::value) {
      TcDotsArgs a;
      a.nks = nks_; a.nbnd = nbnd_; a.npw_pad = hq_.npw_pad; a.nchunk = nchunk_; a.nproj = nproj_; a.nb = nb;
      a.npw = dq_.npw;
      a.x = reinterpret_cast<const float4*>(x);
      a.t = reinterpret_cast<const float4*>(t);
      a.t2 = reinterpret_cast<const float4*>(t2);
      a.ukq = reinterpret_cast<const float4*>(ukq_);
      a.bkq = reinterpret_cast<const float4*>(bkq_);
      a.cpart = cpart; a.spart = spart; a.err = err_; a.jdev = jdev_;
      const size_t sm = tc_dots_smem(nb, tc_nsrc<MODE>(nbnd_, nproj_));
      int rc;
      if ((rc = set_smem(k_tc_dots<MODE>, sm, err))) return rc;
      k_tc_dots<MODE><<<dim3(nks_, nvec, nchunk_), kTcThreads, sm, st_>>>(a);
      LL_CK(cudaGetLastError());
      return LL_OK;
    } else {
      err = "tensor-core projections are FP32-path only";
      return LL_EUNSUPPORTED;
    }
  }

  // t <- t + B c - U S on the tensor cores (FP32 path only; tcproj.cuh): nproj 0 applies P_c
  // alone (the update), x and part give the norm partial.
  int tc_apply(int nvec, int nproj, const cplx<T>* x, cplx<T>* t, double* part, std::string& err) {
    if constexpr (std::is_same<T, float>::value) {
      TcApplyArgs a;
      a.nks = nks_; a.nbnd = nbnd_; a.npw_pad = hq_.npw_pad; a.nchunk = nchunk_; a.nproj = nproj;
      a.nb = tc_nb_ap_;
      a.nks_k = (2 * (nproj + nbnd_) + 15) / 16;
      a.npw = dq_.npw;
      a.x = part ? reinterpret_cast<const float2*>(x) : nullptr;
      a.t = reinterpret_cast<float2*>(t);
      a.ukq = reinterpret_cast<const float2*>(ukq_);
      a.bkq = reinterpret_cast<const float2*>(bkq_);
      a.coef = reinterpret_cast<const float2*>(sp_coef_);
      a.part = part; a.err = err_; a.jdev = jdev_;
      const size_t sm = tc_apply_smem(a.nb, a.nks_k);
      int rc;
      if ((rc = set_smem(k_tc_apply, sm, err))) return rc;
      k_tc_apply<<<dim3(nks_, nvec, nchunk_), kTcThreads, sm, st_>>>(a);
      LL_CK(cudaGetLastError());
      return LL_OK;
    } else {
      err = "tensor-core projections are FP32-path only";
      return LL_EUNSUPPORTED;
    }
  }

  // split per-k path (split.cuh): several CTAs per k-point, chunk partials reduced in order
  template <int N>
  int zfwd_split_n(int nvec, const cplx<T>* in, cplx<T>* out, std::string& err) {
    const int pq = hq_.npw_pad;
    if (metal_) in = img_;   // a metal: the kinetic, KB and norm terms act on the image Q z
    const int lines = (nbnd_ * hq_.ncol_max + kLines - 1) / kLines;
    k_sp_zfwd<T, N><<<dim3(nks_, nvec, lines), kLines, 0, st_>>>(dq_, nbnd_, cbuf_, cb_ncol_, in, kin_, eps_, out);
    const size_t sm_d = (size_t)(std::max(nproj_, nbnd_) + nbnd_) * kTileP * sizeof(cplx<T>);
    const size_t sm_a = (size_t)(nproj_ + nbnd_) * (nbnd_ + kSub) * sizeof(cplx<T>);
    int rc;
    const size_t sm_c = (size_t)nproj_ * nbnd_ * sizeof(cplx<double>);
    if ((rc = set_smem(k_sp_dots<T>, sm_d, err)) || (rc = set_smem(k_sp_coef<T>, sm_c, err)) ||
        (rc = set_smem(k_sp_apply<T>, sm_a, err)))
      return rc;
    if (tc_op_) {
      if ((rc = tc_dots<TC_OP>(nvec, tc_nb_op_, in, out, nullptr, sp_c_, sp_s_, err))) return rc;
    } else {
      k_sp_dots<T><<<dim3(nks_, nvec, nchunk_), 256, sm_d, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, nproj_, in, out,
                                                                  ukq_, bkq_, sp_c_, sp_s_);
    }
    k_sp_coef<T><<<nks_ * nvec, 256, sm_c, st_>>>(nks_, nbnd_, nchunk_, nproj_, dij_, ub_, sp_c_, sp_s_, sp_coef_,
                                                  metal_ ? 1 : 0, md_, zp_, mcorr_);
    if (tc_ap_) {
      if ((rc = tc_apply(nvec, nproj_, in, out, part_, err))) return rc;
    } else {
      k_sp_apply<T><<<dim3(nks_, nvec, nchunk_), 256, sm_a, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, nproj_, in,
                                                                   out, ukq_, bkq_, sp_coef_, part_);
    }
    if (metal_) k_sp_addcorr<<<1, 256, 0, st_>>>(nvec * nks_, nchunk_, mcorr_, part_);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  template <int N>
  int zinv_split_n(int j, std::string& err) {
    const int pq = hq_.npw_pad;
    const size_t sm = (size_t)(2 * nbnd_) * kTileP * sizeof(cplx<T>);
    int rc;
    if ((rc = set_smem(k_sp_start<T>, sm, err))) return rc;
    Coef co{beta_, gamma_, zpart_, err_};
    k_sp_start<T><<<dim3(nks_, nchunk_), 256, sm, st_>>>(jdev_, nks_, nbnd_, pq, dq_.npw, nchunk_, part_, R(), X(), Vp(),
                                                         y_, ukq_, co, tol_, sp_s_, tc_u_ ? 0 : 1);
    if (tc_u_ && (rc = tc_dots<TC_U>(1, tc_nb_u_, nullptr, R(), nullptr, nullptr, sp_s_, err))) return rc;
    // P_c with the chunk-reduced coefficients, tiled (U read once per chunk for all bands),
    // then the axis-3 inverse FFTs over many CTAs per k
    const size_t sm_a = (size_t)nbnd_ * (nbnd_ + kSub) * sizeof(cplx<T>);
    if ((rc = set_smem(k_sp_apply<T>, sm_a, err))) return rc;
    k_sp_coef<T><<<nks_, 256, 0, st_>>>(nks_, nbnd_, nchunk_, 0, dij_, ub_, sp_c_, sp_s_, sp_coef_, metal_ ? 2 : 0,
                                        md_);
    if (tc_ap_) {
      if ((rc = tc_apply(1, 0, nullptr, R(), nullptr, err))) return rc;
    } else {
      k_sp_apply<T><<<dim3(nks_, 1, nchunk_), 256, sm_a, st_>>>(nks_, nbnd_, pq, dq_.npw, nchunk_, 0, nullptr, R(),
                                                                ukq_, bkq_, sp_coef_, nullptr);
    }
    const cplx<T>* rin = metal_image(R(), 1);
    if (!rin) { err = "metal image launch"; return LL_ECUDA; }
    k_zinv<T, N><<<dim3(nks_, 1, zsplit()), 128, 0, st_>>>(dq_, rin, nbnd_, cbuf_, cb_ncol_);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  template <int N>
  int zinv_ph_n(int j, std::string& err) {
    if (split_) return zinv_split_n<N>(j, err);
    const size_t smem = (size_t)bpc_ * hq_.npw_pad * sizeof(cplx<T>) + (size_t)nbnd_ * bpc_ * sizeof(cplx<double>) +
                        red_bytes(256);
    int rc;
    Coef co{beta_, gamma_, zpart_, err_};
    // the per-(k, band group) update, then the axis-3 inverse FFTs, one thread per column line
    if ((rc = set_smem(k_ph_update<T>, smem, err))) return rc;
    k_ph_update<T><<<dim3(nks_, ngrp_), 256, smem, st_>>>(jdev_, dq_, nbnd_, bpc_, part_, R(), X(), Vp(), y_, ukq_, co,
                                                          tol_, md_.keep);
    k_zinv<T, N><<<dim3(nks_, 1, zsplit()), 128, 0, st_>>>(dq_, metal_image(R(), 1), nbnd_, cbuf_, cb_ncol_);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  int launch_zinv_ph(int j, std::string& err) {
    switch (N_) {
      case 12: return zinv_ph_n<12>(j, err);
      case 16: return zinv_ph_n<16>(j, err);
      case 18: return zinv_ph_n<18>(j, err);
      case 24: return zinv_ph_n<24>(j, err);
      case 32: return zinv_ph_n<32>(j, err);
      case 36: return zinv_ph_n<36>(j, err);
      case 48: return zinv_ph_n<48>(j, err);
    }
    return LL_EUNSUPPORTED;
  }

  // CTAs per k-block of the axis-3 inverse FFTs: one column line per thread
  int zsplit() const { return std::max(1, (nbnd_ * std::max(hk_.ncol_max, hq_.ncol_max) + 127) / 128); }
  template <int N>
  int zinv_n(const SphereDev& s, const cplx<T>* in, int nvec) {
    k_zinv<T, N><<<dim3(nks_, nvec, zsplit()), 128, 0, st_>>>(s, in, nbnd_, cbuf_, cb_ncol_);
    return cudaGetLastError() == cudaSuccess ? LL_OK : LL_ECUDA;
  }
  int launch_zinv(const SphereDev& s, const cplx<T>* in, int nvec) {
    switch (N_) {
      case 12: return zinv_n<12>(s, in, nvec);
      case 16: return zinv_n<16>(s, in, nvec);
      case 18: return zinv_n<18>(s, in, nvec);
      case 24: return zinv_n<24>(s, in, nvec);
      case 32: return zinv_n<32>(s, in, nvec);
      case 36: return zinv_n<36>(s, in, nvec);
      case 48: return zinv_n<48>(s, in, nvec);
    }
    return LL_EUNSUPPORTED;
  }
  int groups_for(int norb) const {
    const int target = 4 * nsm_;
    int g = std::max(1, (target + N_ - 1) / N_);
    return std::min(g, norb);
  }
  // Orbital groups of one plane-pass launch (grid N x groups): as many CTAs as fit on the
  // GPU at once for this mode's occupancy, so that the launch is a single wave.
  template <typename K>
  int groups_for_kernel(K kernel, size_t smem, int norb, int& cache, int threads = 128) {
    if (cache == 0) {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
      }
      cache = std::max(1, (occ * nsm_) / N_);
    }
    return std::max(1, std::min(std::min(cache, ngroups_), norb));
  }
  template <int N, int MODE>
  int xy_nm(const SphereDev& s, int norb, int o_off, int dens_vec, std::string& err) {
    const XyChoice c = xy_choice_[MODE];
    if constexpr (N == 24 || N == 32 || N == 36 || N == 48) {
      // every line transform split over a lane pair (xypair.cuh): half the registers per thread.
      // Untuned default: N = 48 only (measured on GB300: faster at N = 48, 16-atom cell pass 2
      // 0.67 -> 0.55 ms per step; slower at N = 32, KB workload pass 1 0.26 -> 0.29 ms)
      const bool pair = xy_pair_ >= 0 ? xy_pair_ == 1 : (c.var >= 0 ? c.var == 1 : N == 48);
      if (pair) return xy_launch<N, MODE>(k_xyp<T, N, MODE>, 4 * N, 2, c.bo, s, norb, o_off, dens_vec, err);
    }
    if constexpr (MODE != XY_STORE) {   // lines pruned to the spheres' extent
      if constexpr (tight_prune(N) > 0)
        if (prune_ == tight_prune(N))
          return xy_launch<N, MODE>(k_xy<T, N, MODE, tight_prune(N)>, 128, 128 / N, c.bo, s, norb, o_off, dens_vec, err);
      if (prune_ == N / 4) return xy_launch<N, MODE>(k_xy<T, N, MODE, N / 4>, 128, 128 / N, c.bo, s, norb, o_off, dens_vec, err);
    }
    return xy_launch<N, MODE>(k_xy<T, N, MODE>, 128, 128 / N, c.bo, s, norb, o_off, dens_vec, err);
  }
  template <int N, int MODE, typename K>
  int xy_launch(K kernel, int threads, int slots, int bo, const SphereDev& s, int norb, int o_off, int dens_vec,
                std::string& err) {
    int B = bo > 0 ? bo : BO<N, MODE>::v;
    XYArgs a;
    a.s = s;
    a.nbnd = nbnd_;
    a.norb = norb;
    a.cb_ncol = cb_ncol_;
    a.o_off = o_off;
    a.dens_vec = dens_vec;
    a.f_ncol = FastDiv((unsigned)cb_ncol_);
    a.f_nrow = FastDiv((unsigned)s.nrow_max);
    a.f_nbnd = FastDiv((unsigned)nbnd_);
    a.f_nks = FastDiv((unsigned)s.nks);
    a.f_pervec = FastDiv((unsigned)(s.nks * nbnd_));
    const int NP = N + 1;
    auto smem_for = [&](int b) {
      size_t m = (size_t)b * cb_ncol_ + (size_t)b * s.nrow_max * NP;
      if (MODE == XY_PASS2) m += (size_t)N * N;
      if (MODE == XY_PASS1_DENS) m += (size_t)slots * N * N;   // per-slot density planes
      m *= sizeof(cplx<T>);
      if (MODE == XY_PASS1 || MODE == XY_PASS1_DENS) m += (size_t)N * N * sizeof(T);
      return m;
    };
    // fewer orbitals per batch where the default batch's tiles exceed shared memory (FP64 at
    // N = 48 on the 16-atom cell), or would keep the SM below the CTA count its registers
    // allow (N = 48: 116 KB for 8 orbitals left one 4-warp CTA per SM)
    if (xy_occ_reg_[MODE] == 0) {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
      }
      xy_occ_reg_[MODE] = std::min(occ, 8);
    }
    const size_t per_sm = 227 * 1024 - 2048 * (size_t)xy_occ_reg_[MODE];
    if (bo > 0) {   // a tuned batch: only the shared-memory limit applies
      while (B > 1 && smem_for(B) > 200 * 1024) --B;
    } else {
      while (B > 1 && (smem_for(B) > 200 * 1024 || smem_for(B) * xy_occ_reg_[MODE] > per_sm)) --B;
    }
    const size_t smem = smem_for(B);
    a.bo = B;
    int rc;
    if ((rc = set_smem(kernel, smem, err))) return rc;
    const int ng = groups_for_kernel(kernel, smem, norb, xy_groups_[MODE], threads);
    a.per_group = (norb + ng - 1) / ng;
    kernel<<<dim3(N, ng), threads, smem, st_>>>(a, cbuf_, vloc_, vpr_, ur_, nprt_, ur_);
    if (MODE == XY_PASS1_DENS) last_ng_ = ng;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { err = std::string("k_xy: ") + cudaGetErrorString(e); return LL_ECUDA; }
    return LL_OK;
  }
  // ---- autotuner of the plane pass ----------------------------------------------------
  // For each mode of the operator's plane pass (pass 1, pass 1 with the density, pass 2) the
  // kernel variant (one thread or a lane pair per line transform) and the orbital batch are
  // chosen by timing whole operator applications on a scratch copy of the starting vector
  // (CUDA events on the chain's stream; one mode at a time, the others at their current
  // choice).  The choice is kept per system shape and device for the whole process, so every
  // chain of one shape in a process uses the same launches (their results agree bit for bit
  // whatever else runs); LL_TUNE=0 keeps the untuned defaults.
  int tune_plane_pass(std::string& err) {
    const char* te = getenv("LL_TUNE");
    if (te && te[0] == '0' && te[1] == 0) return LL_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    char key[256];
    snprintf(key, sizeof(key), "%d/%zu/%d/%d/%d/%d/%d/%d/%d/%d/%d/%d/%d", dev, sizeof(T), N_, nks_, nbnd_,
             hq_.npw_pad, cb_ncol_, hq_.nrow_max, nproj_, (int)split_, xy_pair_, (int)prune_, nsm_);
    {
      std::lock_guard<std::mutex> lock(tune_mutex());
      auto it = tune_cache().find(key);
      if (it != tune_cache().end()) {
        for (int m = 0; m < 3; ++m) xy_choice_[m] = {it->second[2 * m], it->second[2 * m + 1]};
        for (int m = 0; m < 3; ++m) xy_occ_reg_[m] = xy_groups_[m] = 0;
        return LL_OK;
      }
    }
    const long vq = (long)nks_ * nbnd_ * hq_.npw_pad;
    int rc;
    if (!scratch_ && (rc = alloc(&scratch_, 2 * vq))) return rc;
    cudaEvent_t ea, eb;
    LL_CK(cudaEventCreate(&ea));
    LL_CK(cudaEventCreate(&eb));
    auto run = [&](int dens, float* ms) -> int {
      LL_CK(cudaMemcpyAsync(scratch_, y_, vq * sizeof(cplx<T>), cudaMemcpyDeviceToDevice, st_));
      LL_CK(cudaEventRecord(ea, st_));
      int r = op(1, scratch_, scratch_ + vq, dens, err);
      if (r) return r;
      LL_CK(cudaEventRecord(eb, st_));
      LL_CK(cudaEventSynchronize(eb));
      LL_CK(cudaEventElapsedTime(ms, ea, eb));
      return LL_OK;
    };
    float ms = 0.f;
    const bool can_pair = (N_ == 24 || N_ == 32 || N_ == 36 || N_ == 48) && xy_pair_ < 0;
    rc = run(approx_ == LL_APPROX_IPA ? -1 : 0, &ms);   // warm-up: lazy module loads, attributes
    const int modes[3] = {XY_PASS1, XY_PASS1_DENS, XY_PASS2};
    for (int mi = 0; mi < 3 && rc == LL_OK; ++mi) {
      const int mode = modes[mi];
      if (mode != XY_PASS1 && approx_ == LL_APPROX_IPA) break;   // no density without K
      const int dens = mode == XY_PASS1 ? -1 : 0;
      const int bdef = (mode == XY_PASS1) ? 384 / N_ : 256 / N_;
      std::vector<XyChoice> cand;
      for (int var = 0; var <= (can_pair ? 1 : 0); ++var) {
        cand.push_back({var, 0});                             // the occupancy-derived batch
        for (int b : {bdef, std::max(1, bdef / 2)}) cand.push_back({var, b});
      }
      // every candidate timed twice, the rounds interleaved; the fastest of its two times counts
      std::vector<float> tmin(cand.size(), 1e30f);
      for (int rep = 0; rep < 2 && rc == LL_OK; ++rep)
        for (size_t ci = 0; ci < cand.size(); ++ci) {
          xy_choice_[mode] = cand[ci];
          xy_occ_reg_[mode] = xy_groups_[mode] = 0;
          if ((rc = run(dens, &ms)) != LL_OK) break;
          tmin[ci] = std::min(tmin[ci], ms);
        }
      XyChoice pick = cand[0];
      float best = 1e30f;
      for (size_t ci = 0; ci < cand.size(); ++ci)
        if (tmin[ci] < best) { best = tmin[ci]; pick = cand[ci]; }
      xy_choice_[mode] = pick;
      xy_occ_reg_[mode] = xy_groups_[mode] = 0;
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (rc != LL_OK) return rc;
    std::lock_guard<std::mutex> lock(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {   // another chain of this shape tuned meanwhile: use its choice
      for (int m = 0; m < 3; ++m) xy_choice_[m] = {it->second[2 * m], it->second[2 * m + 1]};
      for (int m = 0; m < 3; ++m) xy_occ_reg_[m] = xy_groups_[m] = 0;
    } else {
      std::array<int, 6> v;
      for (int m = 0; m < 3; ++m) v[2 * m] = xy_choice_[m].var, v[2 * m + 1] = xy_choice_[m].bo;
      tune_cache()[key] = v;
    }
    return LL_OK;
  }
  static std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
  }
  static std::map<std::string, std::array<int, 6>>& tune_cache() {
    static std::map<std::string, std::array<int, 6>> c;
    return c;
  }

  // mode 0: operator pass 1 (with the density when dens_vec >= 0); 1: pass 2; 2: store x(r)
  template <int N>
  int xy_n(const SphereDev& s, int norb, int o_off, int dens_vec, int mode, std::string& err) {
    if (mode == 0) return dens_vec >= 0 ? xy_nm<N, XY_PASS1_DENS>(s, norb, o_off, dens_vec, err)
                                        : xy_nm<N, XY_PASS1>(s, norb, o_off, -1, err);
    if (mode == 1) return xy_nm<N, XY_PASS2>(s, norb, o_off, dens_vec, err);
    return xy_nm<N, XY_STORE>(s, norb, o_off, -1, err);
  }
  int launch_xy(const SphereDev& s, int norb, int o_off, int dens_vec, int mode, std::string& err) {
    switch (N_) {
      case 12: return xy_n<12>(s, norb, o_off, dens_vec, mode, err);
      case 16: return xy_n<16>(s, norb, o_off, dens_vec, mode, err);
      case 18: return xy_n<18>(s, norb, o_off, dens_vec, mode, err);
      case 24: return xy_n<24>(s, norb, o_off, dens_vec, mode, err);
      case 32: return xy_n<32>(s, norb, o_off, dens_vec, mode, err);
      case 36: return xy_n<36>(s, norb, o_off, dens_vec, mode, err);
      case 48: return xy_n<48>(s, norb, o_off, dens_vec, mode, err);
    }
    return LL_EUNSUPPORTED;
  }
  template <int N>
  int hxc_n(std::string& err) {
    const T scale = (T)(4.0 / (omega_ * nks_));
    if (nsym_ > 1) {   // the density averaged over the small group of Q, then the same transforms
      k_dens_sym<T><<<4 * nsm_, 256, 0, st_>>>(nprt_, last_ng_, N, scale, nsym_, sym_, ng_);
      k_hxc_fwd<T, N><<<N, 256, 0, st_>>>(ng_, 1, T(1), nr_, ng_);
    } else {
      k_hxc_fwd<T, N><<<N, 256, 0, st_>>>(nprt_, last_ng_, scale, nr_, ng_);
    }
    k_hxc_z<T, N><<<(N * N + 63) / 64, 64, 0, st_>>>(ng_, whart_);
    k_hxc_inv<T, N><<<N, 64, 0, st_>>>(ng_, nr_, fxc_, vpr_);
    LL_CK(cudaGetLastError());
    return LL_OK;
  }
  int launch_hxc(std::string& err) {
    switch (N_) {
      case 12: return hxc_n<12>(err);
      case 16: return hxc_n<16>(err);
      case 18: return hxc_n<18>(err);
      case 24: return hxc_n<24>(err);
      case 32: return hxc_n<32>(err);
      case 36: return hxc_n<36>(err);
      case 48: return hxc_n<48>(err);
    }
    return LL_EUNSUPPORTED;
  }

  template <typename F>
  // Opts the kernel in to `bytes` of dynamic shared memory (static shared memory counts
  // against the same 48 KB default, so the opt-in is made whenever the sum passes it).
  int set_smem(F* fn, size_t bytes, std::string& err) {
    const void* key = reinterpret_cast<const void*>(fn);
    for (auto& e : smem_set_)
      if (e.first == key && e.second >= bytes) return LL_OK;
    cudaFuncAttributes at;
    LL_CK(cudaFuncGetAttributes(&at, fn));
    if (bytes + at.sharedSizeBytes > 227 * 1024) {
      err = "shared-memory tile exceeds 227 KB for this system";
      return LL_EUNSUPPORTED;
    }
    if (bytes + at.sharedSizeBytes > 48 * 1024)
      LL_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    smem_set_.push_back({key, bytes});
    return LL_OK;
  }

  static std::vector<cplx<T>> pad_batch(const double* src, const HostSphere& h, int nb,
                                        const std::vector<double>* kscale = nullptr) {
    std::vector<cplx<T>> out((size_t)h.nks * nb * h.npw_pad, czero<T>());
    size_t pos = 0;
    for (int k = 0; k < h.nks; ++k) {
      const double f = kscale ? (*kscale)[k] : 1.0;
      for (int v = 0; v < nb; ++v)
        for (int i = 0; i < h.npw[k]; ++i, ++pos)
          out[((size_t)k * nb + v) * h.npw_pad + i] = mk((T)(f * src[2 * pos]), (T)(f * src[2 * pos + 1]));
    }
    return out;
  }
  static void unpad_batch(const std::vector<cplx<T>>& in, const HostSphere& h, int nb, double* dst) {
    size_t pos = 0;
    for (int k = 0; k < h.nks; ++k)
      for (int v = 0; v < nb; ++v)
        for (int i = 0; i < h.npw[k]; ++i, ++pos) {
          const cplx<T> c = in[((size_t)k * nb + v) * h.npw_pad + i];
          dst[2 * pos] = (double)c.x;
          dst[2 * pos + 1] = (double)c.y;
        }
  }

  // The u_{vk}(r) grids: own (counted in bytes_, freed with the last chain that uses them) or
  // the donor's.
  int ur_alloc(long count) {
    if (donor_) {
      ur_share_ = donor_->ur_share_;
      ur_ = donor_->ur_;
      return LL_OK;
    }
    void* q = nullptr;
    const size_t nbytes = sizeof(cplx<T>) * (size_t)std::max(1L, count);
    if (cudaMalloc(&q, nbytes) != cudaSuccess) { cudaGetLastError(); return LL_ENOMEM; }
    ur_share_ = std::shared_ptr<void>(q, [](void* a) { cudaFree(a); });
    ur_ = static_cast<cplx<T>*>(q);
    bytes_ += nbytes;
    return LL_OK;
  }

  template <typename U>
  int alloc(U** p, long count) {
    void* q = nullptr;
    const size_t nbytes = sizeof(U) * (size_t)std::max(1L, count);
    if (cudaMalloc(&q, nbytes) != cudaSuccess) { cudaGetLastError(); return LL_ENOMEM; }
    ptrs_.push_back({q, nbytes});
    bytes_ += nbytes;
    *p = static_cast<U*>(q);
    return LL_OK;
  }
  template <typename U>
  void release(U* p) {
    if (!p) return;
    auto it = std::find_if(ptrs_.begin(), ptrs_.end(), [&](const std::pair<void*, size_t>& a) {
      return a.first == (void*)p;
    });
    if (it != ptrs_.end()) {
      cudaFree(p);
      bytes_ -= it->second;
      ptrs_.erase(it);
    }
  }
  int upload_sphere(const HostSphere& h, SphereDev& dsph, std::string& err) {
    int *npw, *ncol, *nrow, *cs;
    int4 *col, *row;
    int rc;
    if ((rc = alloc(&npw, h.nks)) || (rc = alloc(&ncol, h.nks)) || (rc = alloc(&nrow, h.nks)) ||
        (rc = alloc(&cs, (long)h.colstart.size())) || (rc = alloc(&col, (long)h.col.size())) ||
        (rc = alloc(&row, (long)h.row.size())))
      return rc;
    LL_CK(cudaMemcpyAsync(npw, h.npw.data(), h.nks * sizeof(int), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(ncol, h.ncol.data(), h.nks * sizeof(int), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(nrow, h.nrow.data(), h.nks * sizeof(int), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(cs, h.colstart.data(), h.colstart.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(col, h.col.data(), h.col.size() * sizeof(int4), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaMemcpyAsync(row, h.row.data(), h.row.size() * sizeof(int4), cudaMemcpyHostToDevice, st_));
    LL_CK(cudaStreamSynchronize(st_));
    dsph.nks = h.nks;
    dsph.npw_pad = h.npw_pad;
    dsph.ncol_max = h.ncol_max;
    dsph.nrow_max = h.nrow_max;
    dsph.npw = npw;
    dsph.ncol = ncol;
    dsph.nrow = nrow;
    dsph.col = col;
    dsph.colstart = cs;
    dsph.row = row;
    return LL_OK;
  }

  // batch vectors: PH uses [R | X | v_{j-1}], NH uses [v_j w_j | XV XW | v_{j-1} w_{j-1}]
  long vq() const { return (long)nks_ * nbnd_ * hq_.npw_pad; }
  cplx<T>* R() { return vecs_; }
  cplx<T>* X() { return vecs_ + vq(); }
  cplx<T>* Vp() { return vecs_ + 2 * vq(); }
  cplx<T>* Vc() { return vecs_; }
  cplx<T>* Wc() { return vecs_ + vq(); }
  cplx<T>* XV() { return vecs_ + 2 * vq(); }
  cplx<T>* XW() { return vecs_ + 3 * vq(); }
  cplx<T>* VpNH() { return vecs_ + 4 * vq(); }
  cplx<T>* Wp() { return vecs_ + 5 * vq(); }

  cudaStream_t st_ = nullptr;
  int N_ = 0, nks_ = 0, nbnd_ = 0, nproj_ = 0, approx_ = 0, flavour_ = 0, cap_ = 0, nvec_ = 1, ngroups_ = 1;
  int nsm_ = 152;           // SMs of the device
  int xy_groups_[4] = {0, 0, 0, 0};   // plane-pass groups per mode (one wave), 0 = not yet known
  int cb_ncol_ = 0, steps_ = 0, queued_ = 0, spec_cap_ = 0, last_ng_ = 1;
  bool stopped_ = false;
  Profiler prof_;
  std::vector<std::pair<const void*, size_t>> smem_set_;
  double omega_ = 0, q_[3] = {0, 0, 0}, tol_ = 0;
  HostSphere hk_, hq_;
  SphereDev dk_{}, dq_{};
  std::vector<std::pair<void*, size_t>> ptrs_;   // every allocation and its size
  std::shared_ptr<void> ur_share_;               // the u_{vk}(r) grids, possibly shared
  std::vector<double> kscale_;                   // sqrt(w_k nks / sum w): folded into u_k
  std::vector<double> rowscale_;                 // [nks][nbnd] kscale_ times sqrt(f_vk) (a metal)
  bool metal_ = false;                           // occupations given (Sec. 2.6)
  std::vector<double> mtab_;                     // the MetalDev tables on the host
  double* mc_ = nullptr;                         // ... and on the device
  MetalDev md_{nullptr, nullptr, nullptr, nullptr};
  cplx<T>* img_ = nullptr;                       // the image Q z of the operator's input (a metal)
  cplx<double>* zp_ = nullptr;                   // Z = U^H z of that input, [nvec][nks][nbnd][nbnd]
  double* mcorr_ = nullptr;                      // the metal's norm term per (vector, k), split path
  std::vector<int> sym_host_;                    // small group of Q on the grid, [nsym][9]
  int nsym_ = 1;
  int* sym_ = nullptr;
  uint64_t gs_hash_ = 0;                         // ground_state_hash of the inputs (0: not shareable)
  Chain<T>* donor_ = nullptr;                    // during create_shared only
  size_t bytes_ = 0;
  T *whart_ = nullptr, *kin_ = nullptr, *vloc_ = nullptr, *fxc_ = nullptr;
  double *rho_ = nullptr, *eps_ = nullptr, *dij_ = nullptr, *part_ = nullptr, *beta_ = nullptr;
  cplx<T> *uk_ = nullptr, *ukq_ = nullptr, *bkq_ = nullptr, *ur_ = nullptr, *cbuf_ = nullptr, *nprt_ = nullptr;
  cplx<T> *nr_ = nullptr, *ng_ = nullptr, *vpr_ = nullptr, *y_ = nullptr, *vecs_ = nullptr;
  cplx<T>* scratch_ = nullptr;
  cplx<double> *spart_ = nullptr, *gamma_ = nullptr, *z_ = nullptr, *zpart_ = nullptr, *spec_out_ = nullptr;
  ExtrapTail* tail_ = nullptr;   // continuation constants of the coefficients (spectrum)
  int* jdev_ = nullptr;          // device step counter of the pseudo-Hermitian recursion
  bool use_graphs_ = true;       // replay captured steps (LL_GRAPHS=0 in the environment: eager)
  bool eager_done_[2] = {false, false};
  cudaGraphExec_t graph_[2] = {nullptr, nullptr};   // one captured step per parity of j
  bool split_ = false;      // per-k work split over chunks of plane waves (split.cuh)
  int xy_occ_reg_[4] = {0, 0, 0, 0};   // CTAs per SM the plane pass's registers allow, per mode
  int xy_pair_ = -1;                   // LL_XY_PAIR: 1 lane pairs for every even N, 0 never, -1 not forced
  int prune_ = 0;                      // line transforms pruned to |m| <= prune_ (0: unpruned)
  struct XyChoice { int var; int bo; };    // plane-pass kernel (0 k_xy, 1 k_xyp) and orbital batch
  XyChoice xy_choice_[4] = {{-1, 0}, {-1, 0}, {-1, 0}, {-1, 0}};   // per mode; -1 / 0: the untuned default
  bool tc_op_ = false, tc_u_ = false, tc_u2_ = false;   // split-path dot blocks on the tensor cores
  bool tc_ap_ = false;                                    // split-path projections applied on the tensor cores
  int tc_nb_op_ = 32, tc_nb_u_ = 32, tc_nb_ap_ = 32;      // N of those MMAs (Bop rows, padded to 32)
  int nchunk_ = 1;          // plane-wave chunks per k on the split path
  int bpc_ = 1, ngrp_ = 1;  // bands per CTA of the per-k kernels, band groups per k
  int npk_ = 1;             // partial sums per k of the Lanczos scalars (ngrp_, or nchunk_ split)
  cplx<double> *sp_s_ = nullptr, *sp_c_ = nullptr, *ub_ = nullptr;   // chunk partials of U^H r, B^H x; U^H B
  cplx<T>* sp_coef_ = nullptr;   // reduced KB and P_c coefficients per (vector, k) of the split apply
  double* spec_w_ = nullptr;
  int *map_ = nullptr, *err_ = nullptr;
};

}  // namespace ll
