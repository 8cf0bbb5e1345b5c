// C ABI of libll.so: argument checks, error strings, dispatch to the precision-specific
// chain (FP64 or FP32).  See include/ll.h for the contract of every entry point.
#include <cuda.h>
#include <string.h>

#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "chain.cuh"

struct ll_handle {
  ll::ChainBase* chain = nullptr;
  cudaStream_t stream = nullptr;
  int device = 0;
};

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
}  // namespace

// ---------------------------------------------------------------------------------------
// FMA throughput of the device: every thread runs 8 independent chains x <- x*m + c for
// `iters` iterations (8 * iters FMAs, 2 flops each).  The multiplier is 1 - 2^-20 and the
// addend small, so the chains stay finite; one store per thread, predicated on a value that
// never occurs, keeps the work from being removed.
namespace {
template <typename T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T m, T c, T* sink) {
  T x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = T(threadIdx.x + q);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], m, c);
  }
  T t = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) t += x[q];
  if (t == T(-1.25)) sink[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

template <typename T>
int fma_peak(double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(LL_ECUDA, "ll_fma_peak: device query");
  const int blocks = sms * 8, threads = 256, iters = sizeof(T) == 4 ? 16384 : 1024;
  T* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, sizeof(T) * blocks * threads) != cudaSuccess) return fail(LL_ENOMEM, "ll_fma_peak: allocation");
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T m = T(1) - T(1) / T(1 << 20), c = T(1) / T(1 << 10);
  k_fma_peak<T><<<blocks, threads, 0, st>>>(iters / 8, m, c, sink);   // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_peak<T><<<blocks, threads, 0, st>>>(iters, m, c, sink);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    best = ms < best ? ms : best;
  }
  cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return fail(LL_ECUDA, std::string("ll_fma_peak: ") + cudaGetErrorString(e));
  *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return LL_OK;
}
}  // namespace


extern "C" {

const char* ll_last_error(void) { return g_err.c_str(); }
const char* ll_version(void) { return "ll-gb300 1.0 (sm_103a)"; }

int ll_fma_peak(int precision, double* tflops, void* stream) {
  if (!tflops) return fail(LL_EINVAL, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (precision == LL_PREC_FP32) return fma_peak<float>(tflops, st);
  if (precision == LL_PREC_FP64) return fma_peak<double>(tflops, st);
  return fail(LL_EINVAL, "bad precision");
}

int ll_create(const ll_system_desc* desc, void* stream, ll_handle** out) {
  if (!desc || !out) return fail(LL_EINVAL, "null descriptor or output");
  *out = nullptr;
  if (desc->precision != LL_PREC_FP64 && desc->precision != LL_PREC_FP32) return fail(LL_EINVAL, "bad precision");
  ll_handle* h = new (std::nothrow) ll_handle();
  if (!h) return fail(LL_ENOMEM, "host allocation");
  h->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  h->chain = (desc->precision == LL_PREC_FP64) ? ll::make_chain_f64() : ll::make_chain_f32();
  std::string err;
  int rc = h->chain->create(desc, h->stream, err);
  if (rc != LL_OK) {
    delete h->chain;
    delete h;
    return fail(rc, "ll_create: " + err);
  }
  *out = h;
  return LL_OK;
}

int ll_create_sharing(const ll_system_desc* desc, ll_handle* share, void* stream, ll_handle** out) {
  if (!desc || !out || !share) return fail(LL_EINVAL, "null descriptor, sharing handle or output");
  *out = nullptr;
  if (desc->precision != LL_PREC_FP64 && desc->precision != LL_PREC_FP32) return fail(LL_EINVAL, "bad precision");
  ll_handle* h = new (std::nothrow) ll_handle();
  if (!h) return fail(LL_ENOMEM, "host allocation");
  h->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&h->device);
  if (share->stream && share->stream != h->stream) cudaStreamSynchronize(share->stream);   // its grids are built
  h->chain = (desc->precision == LL_PREC_FP64) ? ll::make_chain_f64() : ll::make_chain_f32();
  std::string err;
  int rc = h->chain->create_shared(desc, h->stream, share->chain, err);
  if (rc != LL_OK) {
    delete h->chain;
    delete h;
    return fail(rc, "ll_create_sharing: " + err);
  }
  *out = h;
  return LL_OK;
}

int ll_destroy(ll_handle* h) {
  if (!h) return LL_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  delete h->chain;
  delete h;
  return LL_OK;
}

int ll_lanczos(ll_handle* h, int n_steps, double* alpha, double* beta, double* gamma, double* z, int* steps_done) {
  if (!h) return fail(LL_EINVAL, "null handle");
  std::string err;
  int done = 0;
  int rc = h->chain->lanczos(n_steps, beta, gamma, z, &done, err);
  if (steps_done) *steps_done = done;
  if (alpha)
    for (int i = 0; i < done; ++i) alpha[i] = 0.0;
  return rc == LL_OK ? LL_OK : fail(rc, "ll_lanczos: " + err);
}

static bool extrap_args_ok(int m, int kind, int m_total) {
  if (kind == LL_EXTRAP_NO) return true;
  if (kind != LL_EXTRAP_CONSTANT && kind != LL_EXTRAP_OSC) return false;
  if (m_total < m || m_total > LL_EXTRAP_MAX) return false;
  return m >= (kind == LL_EXTRAP_OSC ? 4 : 2);
}

int ll_lanczos_spectrum(ll_handle* h, int m, const double* omega_ev, int n_omega, double eta_ev, double* chi,
                        double* eps_inv, double* eps) {
  if (!h || !omega_ev || n_omega < 1) return fail(LL_EINVAL, "bad spectrum arguments");
  std::string err;
  int rc = h->chain->spectrum(m, LL_EXTRAP_NO, 0, omega_ev, n_omega, eta_ev, chi, eps_inv, eps, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_lanczos_spectrum: " + err);
}

int ll_lanczos_spectrum_x(ll_handle* h, int m, int kind, int m_total, const double* omega_ev, int n_omega,
                          double eta_ev, double* chi, double* eps_inv, double* eps) {
  if (!h || !omega_ev || n_omega < 1) return fail(LL_EINVAL, "bad spectrum arguments");
  const int mm = (m <= 0 || m > h->chain->steps()) ? h->chain->steps() : m;
  if (!extrap_args_ok(mm, kind, m_total)) return fail(LL_EINVAL, "bad extrapolation arguments");
  std::string err;
  int rc = h->chain->spectrum(m, kind, m_total, omega_ev, n_omega, eta_ev, chi, eps_inv, eps, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_lanczos_spectrum_x: " + err);
}

static int spectrum_impl(const double* beta, const double* gamma, const double* z, int m, int kind, int m_total,
                         double omega_cell, const double* q_cart, const double* omega_ev, int n_omega, double eta_ev,
                         double* chi, double* eps_inv, double* eps, void* stream) {
  if (!beta || !gamma || !z || m < 1 || !q_cart || !omega_ev || n_omega < 1 || !(omega_cell > 0))
    return fail(LL_EINVAL, "bad spectrum arguments");
  if (!extrap_args_ok(m, kind, m_total)) return fail(LL_EINVAL, "bad extrapolation arguments");
  if (kind == LL_EXTRAP_NO) m_total = m;
  const double q2 = q_cart[0] * q_cart[0] + q_cart[1] * q_cart[1] + q_cart[2] * q_cart[2];
  if (!(q2 > 0)) return fail(LL_EINVAL, "Q = 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const double ha = 27.211386245988;
  std::vector<double> w(n_omega);
  for (int i = 0; i < n_omega; ++i) w[i] = omega_ev[i] / ha;
  double *db = nullptr, *dw = nullptr;
  ll::cplx<double> *dg = nullptr, *dz = nullptr, *dout = nullptr;
  ll::ExtrapTail* dt = nullptr;
  auto cleanup = [&]() { cudaFree(db); cudaFree(dw); cudaFree(dg); cudaFree(dz); cudaFree(dout); cudaFree(dt); };
  if (cudaMalloc(&db, m * sizeof(double)) != cudaSuccess || cudaMalloc(&dg, m * sizeof(ll::cplx<double>)) != cudaSuccess ||
      cudaMalloc(&dz, m * sizeof(ll::cplx<double>)) != cudaSuccess || cudaMalloc(&dw, n_omega * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dout, 3L * n_omega * sizeof(ll::cplx<double>)) != cudaSuccess ||
      cudaMalloc(&dt, sizeof(ll::ExtrapTail)) != cudaSuccess) {
    cleanup();
    return fail(LL_ENOMEM, "ll_spectrum: device allocation");
  }
  cudaMemcpyAsync(db, beta, m * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dg, gamma, m * sizeof(ll::cplx<double>), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dz, z, m * sizeof(ll::cplx<double>), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(dw, w.data(), n_omega * sizeof(double), cudaMemcpyHostToDevice, st);
  if (m_total > m) ll::k_extrap_tail<<<1, 256, 0, st>>>(m, kind, db, dg, dt);
  ll::k_spectrum<<<(n_omega + 127) / 128, 128, 0, st>>>(m, m_total, m_total > m ? dt : nullptr, db, dg, dz, n_omega,
                                                         dw, eta_ev / ha, 4.0 / omega_cell,
                                                         4.0 * 3.14159265358979323846 / q2, dout, dout + n_omega,
                                                         dout + 2L * n_omega);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    if (chi) cudaMemcpyAsync(chi, dout, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
    if (eps_inv) cudaMemcpyAsync(eps_inv, dout + n_omega, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
    if (eps) cudaMemcpyAsync(eps, dout + 2L * n_omega, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
    e = cudaStreamSynchronize(st);
  }
  cleanup();
  if (e != cudaSuccess) return fail(LL_ECUDA, std::string("ll_spectrum: ") + cudaGetErrorString(e));
  return LL_OK;
}

int ll_spectrum(const double* beta, const double* gamma, const double* z, int m, double omega_cell, const double* q_cart,
                const double* omega_ev, int n_omega, double eta_ev, double* chi, double* eps_inv, double* eps,
                void* stream) {
  return spectrum_impl(beta, gamma, z, m, LL_EXTRAP_NO, m, omega_cell, q_cart, omega_ev, n_omega, eta_ev, chi, eps_inv,
                       eps, stream);
}

int ll_spectrum_x(const double* beta, const double* gamma, const double* z, int m, int kind, int m_total,
                  double omega_cell, const double* q_cart, const double* omega_ev, int n_omega, double eta_ev,
                  double* chi, double* eps_inv, double* eps, void* stream) {
  return spectrum_impl(beta, gamma, z, m, kind, m_total, omega_cell, q_cart, omega_ev, n_omega, eta_ev, chi, eps_inv,
                       eps, stream);
}

// ---------------------------------------------------------------------------------------
// Allocation-free spectrum.  The device staging area lives in one file-scope array that
// every GPU loading the library holds until exit; host code reaches it only through the
// address cudaGetSymbolAddress returns for the current device (the symbol itself is a
// host-side stand-in).  Layout: beta[MAX_COEF] | gamma[MAX_COEF] | z[MAX_COEF] |
// omega[MAX_OMEGA] | chi, eps_inv, eps [MAX_OMEGA each].
namespace {
constexpr int kStaticMaxCoef = LL_SPECTRUM_STATIC_MAX_COEF;
constexpr int kStaticMaxOmega = LL_SPECTRUM_STATIC_MAX_OMEGA;
constexpr size_t kOffGamma = sizeof(double) * kStaticMaxCoef;
constexpr size_t kOffZ = kOffGamma + sizeof(ll::cplx<double>) * kStaticMaxCoef;
constexpr size_t kOffW = kOffZ + sizeof(ll::cplx<double>) * kStaticMaxCoef;
constexpr size_t kOffOut = kOffW + sizeof(double) * kStaticMaxOmega;
constexpr size_t kStaticBytes = kOffOut + 3 * sizeof(ll::cplx<double>) * kStaticMaxOmega;

static __device__ __align__(256) unsigned char g_spectrum_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
// The looked-up address per device, tagged with the id of the context it was looked up in: a
// context destroyed and re-created (cudaDeviceReset, a driver-level context switch) gets a new
// id, and the address is looked up again in the new context.
struct StaticSlot { unsigned long long ctx_id; unsigned char* addr; };
StaticSlot g_static_slot[kMaxDevices] = {};

typedef CUresult (*PFN_ctx_get_current)(CUcontext*);
typedef CUresult (*PFN_ctx_get_id)(CUcontext, unsigned long long*);

// Id of the context current on this thread (0 when none is current yet).
int current_ctx_id(unsigned long long* id, std::string& err) {
  static PFN_ctx_get_current get_current = nullptr;
  static PFN_ctx_get_id get_id = nullptr;
  if (!get_current || !get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e1 != cudaSuccess || e2 != cudaSuccess || !f1 || !f2 || q1 != cudaDriverEntryPointSuccess ||
        q2 != cudaDriverEntryPointSuccess) {
      err = "driver entry points cuCtxGetCurrent/cuCtxGetId unavailable";
      return LL_ECUDA;
    }
    get_current = reinterpret_cast<PFN_ctx_get_current>(f1);
    get_id = reinterpret_cast<PFN_ctx_get_id>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS) { err = "cuCtxGetCurrent failed"; return LL_ECUDA; }
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) { err = "cuCtxGetId failed"; return LL_ECUDA; }
  return LL_OK;
}

// Device address of the staging array in the current device's current context.  The lookup
// runs once per device and context: on the first call on a device (which also makes the
// runtime initialise that device's primary context) and again after the context changed.
int static_scratch(unsigned char** out, std::string& err) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return LL_ECUDA; }
  if (dev < 0 || dev >= kMaxDevices) { err = "device ordinal out of range"; return LL_EUNSUPPORTED; }
  std::lock_guard<std::mutex> lock(g_static_mu);
  unsigned long long id = 0;
  int rc = current_ctx_id(&id, err);
  if (rc != LL_OK) return rc;
  StaticSlot& slot = g_static_slot[dev];
  if (id == 0 || slot.addr == nullptr || slot.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
    if (e != cudaSuccess || !p) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return LL_ECUDA;
    }
    if (id == 0) {   // no context was current before the lookup; the runtime has made one now
      rc = current_ctx_id(&id, err);
      if (rc != LL_OK) return rc;
    }
    slot.ctx_id = id;
    slot.addr = static_cast<unsigned char*>(p);
  }
  *out = slot.addr;
  return LL_OK;
}

__global__ void k_ev_to_ha(int n, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w[i] = w[i] / 27.211386245988;
}
}  // namespace

int ll_spectrum_static(const double* beta, const double* gamma, const double* z, int m, double omega_cell,
                       const double* q_cart, const double* omega_ev, int n_omega, double eta_ev, double* chi,
                       double* eps_inv, double* eps, void* stream) {
  if (!beta || !gamma || !z || m < 1 || !q_cart || !omega_ev || n_omega < 1 || !(omega_cell > 0))
    return fail(LL_EINVAL, "bad spectrum arguments");
  if (m > kStaticMaxCoef)
    return fail(LL_EINVAL, "ll_spectrum_static: " + std::to_string(m) + " coefficients exceed the static limit of " +
                               std::to_string(kStaticMaxCoef));
  if (n_omega > kStaticMaxOmega)
    return fail(LL_EINVAL, "ll_spectrum_static: " + std::to_string(n_omega) +
                               " frequencies exceed the static limit of " + std::to_string(kStaticMaxOmega));
  const double q2 = q_cart[0] * q_cart[0] + q_cart[1] * q_cart[1] + q_cart[2] * q_cart[2];
  if (!(q2 > 0)) return fail(LL_EINVAL, "Q = 0");
  std::string err;
  unsigned char* base = nullptr;
  int rc = static_scratch(&base, err);
  if (rc != LL_OK) return fail(rc, "ll_spectrum_static: " + err);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* db = reinterpret_cast<double*>(base);
  ll::cplx<double>* dg = reinterpret_cast<ll::cplx<double>*>(base + kOffGamma);
  ll::cplx<double>* dz = reinterpret_cast<ll::cplx<double>*>(base + kOffZ);
  double* dw = reinterpret_cast<double*>(base + kOffW);
  ll::cplx<double>* dout = reinterpret_cast<ll::cplx<double>*>(base + kOffOut);
  cudaError_t e = cudaMemcpyAsync(db, beta, m * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, gamma, m * sizeof(ll::cplx<double>), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dz, z, m * sizeof(ll::cplx<double>), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, omega_ev, n_omega * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_ev_to_ha<<<(n_omega + 127) / 128, 128, 0, st>>>(n_omega, dw);
    ll::k_spectrum<<<(n_omega + 127) / 128, 128, 0, st>>>(m, m, nullptr, db, dg, dz, n_omega, dw, eta_ev / 27.211386245988,
                                                           4.0 / omega_cell, 4.0 * 3.14159265358979323846 / q2, dout,
                                                           dout + kStaticMaxOmega, dout + 2L * kStaticMaxOmega);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && chi)
    e = cudaMemcpyAsync(chi, dout, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && eps_inv)
    e = cudaMemcpyAsync(eps_inv, dout + kStaticMaxOmega, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && eps)
    e = cudaMemcpyAsync(eps, dout + 2L * kStaticMaxOmega, n_omega * sizeof(ll::cplx<double>), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(LL_ECUDA, std::string("ll_spectrum_static: ") + cudaGetErrorString(e));
  return LL_OK;
}

// f-sum printout (Sec. 2.1): the trapezoid first moment of the loss function over the grid,
// one block, every thread a strided partial, the partials summed in a fixed order.
namespace {
__global__ void k_fsum(int n, const double* __restrict__ w_ev, const ll::cplx<double>* __restrict__ ei,
                       double* __restrict__ out) {
  __shared__ double part[256];
  const double ha = 27.211386245988;
  double s = 0.0;
  for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) {
    const double w0 = w_ev[i] / ha, w1 = w_ev[i + 1] / ha;
    s += 0.5 * (w0 * -ei[i].y + w1 * -ei[i + 1].y) * (w1 - w0);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) t += part[i];
    out[0] = t;
  }
}
}  // namespace

int ll_fsum(const double* omega_ev, const double* eps_inv, int n_omega, double nelec, double omega_cell,
            double* moment, double* expected, void* stream) {
  if (!omega_ev || !eps_inv || n_omega < 2 || !(omega_cell > 0) || !(nelec >= 0) || !moment)
    return fail(LL_EINVAL, "bad f-sum arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *dw = nullptr, *de = nullptr, *dout = nullptr;
  cudaError_t e = cudaMallocAsync(&dw, n_omega * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&de, 2 * (size_t)n_omega * sizeof(double), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dout, sizeof(double), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dw, omega_ev, n_omega * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(de, eps_inv, 2 * (size_t)n_omega * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_fsum<<<1, 256, 0, st>>>(n_omega, dw, reinterpret_cast<const ll::cplx<double>*>(de), dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(moment, dout, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dw) cudaFreeAsync(dw, st);
  if (de) cudaFreeAsync(de, st);
  if (dout) cudaFreeAsync(dout, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(LL_ECUDA, std::string("ll_fsum: ") + cudaGetErrorString(e));
  if (expected) *expected = 0.5 * 3.14159265358979323846 * 4.0 * 3.14159265358979323846 * nelec / omega_cell;
  return LL_OK;
}

int ll_apply(ll_handle* h, int upper, const double* x, double* out) {
  if (!h || !x || !out) return fail(LL_EINVAL, "bad apply arguments");
  std::string err;
  int rc = h->chain->apply(upper, x, out, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_apply: " + err);
}

int ll_get_map(ll_handle* h, int* map_out) {
  if (!h || !map_out) return fail(LL_EINVAL, "bad arguments");
  std::string err;
  int rc = h->chain->get_map(map_out, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_get_map: " + err);
}

int ll_get_start(ll_handle* h, double* y_out) {
  if (!h || !y_out) return fail(LL_EINVAL, "bad arguments");
  std::string err;
  int rc = h->chain->get_start(y_out, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_get_start: " + err);
}

int ll_profile(ll_handle* h, int enable) {
  if (!h) return fail(LL_EINVAL, "null handle");
  std::string err;
  int rc = h->chain->profile(enable, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_profile: " + err);
}

int ll_profile_read(ll_handle* h, double* ms, long long* launches, long long* total) {
  if (!h) return fail(LL_EINVAL, "null handle");
  std::string err;
  int rc = h->chain->profile_read(ms, launches, total, err);
  return rc == LL_OK ? LL_OK : fail(rc, "ll_profile_read: " + err);
}

int ll_bytes(ll_handle* h, size_t* bytes) {
  if (!h || !bytes) return fail(LL_EINVAL, "bad arguments");
  *bytes = h->chain->bytes();
  return LL_OK;
}

int ll_footprint(const ll_system_desc* d, size_t* bytes) {
  if (!d || !bytes || !d->npw_k || !d->npw_kq || d->nks < 1 || d->nbnd < 1 || d->nfft < 1)
    return fail(LL_EINVAL, "bad footprint arguments");
  const size_t elem = (d->precision == LL_PREC_FP64) ? 16 : 8;
  int mk = 1, mq = 1;
  for (int k = 0; k < d->nks; ++k) {
    mk = d->npw_k[k] > mk ? d->npw_k[k] : mk;
    mq = d->npw_kq[k] > mq ? d->npw_kq[k] : mq;
  }
  const size_t pk = (mk + 3) / 4 * 4, pq = (mq + 3) / 4 * 4;
  const size_t n3 = (size_t)d->nfft * d->nfft * d->nfft;
  const size_t nvec = (d->flavour == LL_FLAVOUR_NH) ? 2 : 1;
  const size_t vq = (size_t)d->nks * d->nbnd * pq;
  const size_t orb = (size_t)d->nks * d->nbnd;
  // columns per sphere are at most the sphere size; bounded by pq for the estimate
  const size_t cb = nvec * orb * d->nfft * pq;
  // density slot planes: 4 per SM of the current device (152 where none can be queried)
  int nsm = 152;
  {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess)
      nsm = std::max(nsm, n);
    cudaGetLastError();
  }
  const size_t ngroups = (4 * (size_t)nsm + d->nfft - 1) / d->nfft;
  // vectors: 3 nvec Lanczos vectors, nvec partial copies, y, U_{k+Q}, and the 2-vector scratch
  // of the plane-pass tuner and ll_apply
  size_t b = elem * (vq * (3 * nvec + nvec + 2 + 2) + orb * pk + orb * n3 + cb + ngroups * n3 + 3 * n3 +
                     (size_t)d->nks * d->nproj * pq);
  // Lanczos partials: up to max(bands, plane-wave chunks) per k and step (band groups or the
  // split path), and the split path's chunk partials and coefficient blocks
  const size_t npk = (size_t)std::max(d->nbnd, (int)((pq + 511) / 512));
  const size_t pairs = (size_t)(d->nproj + d->nbnd) * d->nbnd;
  b += (elem / 2) * (2 * n3 + (size_t)d->nks * pq) + 8 * n3 +
       40 * (size_t)(d->max_steps + 2) * (d->nks * npk + 2) + 48 * nvec * (size_t)d->nks * npk * pairs;
  if (d->occ_k) b += 32 * (size_t)d->nks * d->nbnd * d->nbnd;   // the metal's projector tables
  *bytes = b;
  return LL_OK;
}

}  // extern "C"
