/* C ABI of the GB300 Liouville-Lanczos library (libll.so).
 *
 * The library applies the Liouvillian of time-dependent density-functional perturbation
 * theory, in the standard batch representation, to a batch of plane-wave response orbitals
 * {x_{v,k+Q}} and runs the Lanczos recursions whose coefficients give the charge-density
 * susceptibility chi(Q, omega) and the inverse dielectric function at finite momentum
 * transfer Q (Timrov et al., turboEELS, Sec. 2; Eqs. 10, 23-33).
 *
 * Conventions
 *   - Every function returns an ll_status; nothing throws across the ABI.  After a failure
 *     ll_last_error() returns a message for the calling thread.
 *   - Hartree atomic units throughout, except the frequency grid and broadening of the
 *     spectrum calls (eV, as in the post-processing input of Sec. 3.3).
 *   - Complex numbers are interleaved (re, im) doubles; arrays are C-contiguous.
 *   - Host pointers unless a name ends in _dev.  Input arrays are copied by ll_create; the
 *     caller may free them afterwards.  Output arrays are caller-owned.
 *   - Streams are cudaStream_t passed as void* (NULL = the legacy default stream).
 *   - One handle drives one chain on one device; calls on one handle must not overlap.
 */
#ifndef LL_H
#define LL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LL_OK = 0,
  LL_EINVAL = 1,        /* an argument or an input array is malformed                    */
  LL_ENOMEM = 2,        /* device allocation failed                                      */
  LL_EBREAKDOWN = 3,    /* Lanczos breakdown (|s| or beta^2 below tolerance)             */
  LL_ENOTPD = 4,        /* pseudo-Hermitian metric not positive (D or D+K indefinite)     */
  LL_ETIMEOUT = 5,      /* a bounded device wait gave up                                 */
  LL_ECUDA = 6,         /* a CUDA runtime call failed                                    */
  LL_PENDING = 7,
  LL_ENOTFOUND = 8,
  LL_EUNSUPPORTED = 9,  /* valid input outside what this build implements                */
  LL_ECANCELED = 10     /* the job was cancelled (ll_cancel)                             */
} ll_status;

enum { LL_APPROX_IPA = 0, LL_APPROX_RPA = 1, LL_APPROX_TDDFT = 2 };   /* Sec. 3.2 */
enum { LL_FLAVOUR_PH = 0, LL_FLAVOUR_NH = 1 };                          /* Sec. 2.5 */
enum { LL_PREC_FP64 = 0, LL_PREC_FP32 = 1 };

typedef struct ll_handle ll_handle;

/* Ground state and response set-up of one chain (the data pw.x hands to turbo_eels.x,
 * Sec. 3.1, plus the turbo_eels.x input of Sec. 3.2). */
typedef struct {
  double lattice[3][3];     /* rows a_i, bohr                                              */
  int nfft;                 /* FFT grid N (N^3 points along a_i); 12,16,18,24,32,36,48      */
  int nks;                  /* k-points, weights 1/nks                                     */
  int nbnd;                 /* occupied bands per k (<= 32)                                */
  int nproj;                /* KB projectors per k (0 allowed)                             */
  double q_cart[3];         /* momentum transfer Q (bohr^-1); Q + G != 0 on the grid       */
  const double* kcart;      /* [nks][3]                                                    */
  const int* npw_k;         /* [nks] sphere sizes of k                                     */
  const int* miller_k;      /* [sum npw_k][3], each sphere lexicographic in (m1,m2,m3)     */
  const int* npw_kq;        /* [nks] sphere sizes of k+Q                                   */
  const int* miller_kq;     /* [sum npw_kq][3]                                             */
  const double* u_k;        /* complex, per k [nbnd][npw_k[k]] concatenated: u_{vk}(G)    */
  const double* u_kq;       /* complex, per k [nbnd][npw_kq[k]]: occupied states at k+Q   */
  const double* eps_k;      /* [nks][nbnd] eigenvalues eps_{vk} (Ha)                       */
  const double* vloc_r;     /* [N][N][N] (index j1,j2,j3) total Kohn-Sham local potential  */
  const double* rho_r;      /* [N][N][N] ground-state density (bohr^-3)                    */
  const double* beta_kq;    /* complex, per k [nproj][npw_kq[k]]: beta_p(k+Q+G)            */
  const double* dij;        /* [nproj] KB strengths D_p (Ha)                               */
  int approx;               /* LL_APPROX_*                                                 */
  int flavour;              /* LL_FLAVOUR_*                                                */
  int precision;            /* LL_PREC_*: FP64 everywhere, or FP32 orbitals/FFTs with FP64
                               Lanczos scalars                                             */
  int max_steps;            /* capacity of the device coefficient arrays                   */
  int where;                /* LL_WHERE_HOST (0) or LL_WHERE_DEVICE (1): where u_k, u_kq,
                               beta_kq, vloc_r and rho_r live.  Device arrays (e.g. a torch
                               CUDA tensor's data_ptr()) must be on the current device and
                               stay untouched until ll_create returns; they are read on the
                               device (no host copy).  The index arrays (npw, miller), kcart,
                               eps_k and dij are always host arrays.                         */
  /* k-point symmetry by the small group of Q (Sec. 2.6).  With kweight (host, [nks], > 0) the
   * k-points are the representatives of the stars of a full mesh with these star sizes: every
   * sum over k of the recursions is the weighted sum (the library folds sqrt(w_k nks / sum w)
   * into u_k).  With nsym > 1, sym (host, [nsym][3][3] int, the identity among them) holds
   * the operations of the small group of Q on the FFT grid indices, (j1, j2, j3) -> M j mod N
   * for the grid points r_j = sum_i (j_i/N) a_i, and the response density is averaged over
   * them before v'_HXC is formed.  NULL / 0: the plain full-mesh sums.                      */
  const double* kweight;
  int nsym;
  const int* sym;
  /* Metals by smearing (Sec. 2.6: the projector on empty states redefined, fractional
   * occupations as weights in the band sums).  With occ_k (host, [nks][nbnd], each in [0, 1])
   * the bands are the partially or fully occupied ones: occ_k[k][v] = f_vk weights band v of k
   * in the response density (the library folds sqrt(f_vk) into u_k), occ_kq (host,
   * [nks][nbnd]) holds the occupations f_m of the states u_kq and eps_kq (host, [nks][nbnd],
   * Ha) their eigenvalues (u_kq must be eigenvectors of H_{k+Q}).  Each pair of levels is
   * given to its direction of positive transition energy: per band v the projector on empty
   * states keeps u_m with weight c_mv = max(1 - f_m/f_v, 0) (0 for f_v = 0, and 0 below
   * LL_METAL_CMIN), the Lanczos vectors keep the states with c_mv > 0, and the scalar
   * products carry the metric weight 1/c_mv on them.  Every state of k+Q beyond the nbnd given
   * must lie above every occupied level of k.  The response is for Q + G != 0 (no Fermi-level
   * shift).  NULL: an insulator (every band full).  Both per-k paths (fused, and split
   * over plane-wave chunks with the tensor-core projections) take metals.                   */
  const double* occ_k;
  const double* occ_kq;
  const double* eps_kq;
} ll_system_desc;

#define LL_METAL_CMIN 1e-6

enum { LL_WHERE_HOST = 0, LL_WHERE_DEVICE = 1 };

/* Builds the device state of one chain (Sec. 2.4-2.5): index maps (sphere(k+Q) -> sphere(k)
 * intersection, column/plane tables), u_{vk}(r) grids, f_xc(n0), the Hartree kernel
 * 4 pi/|Q+G|^2, the starting vector y = P_c u (Eq. 28) and, for the pseudo-Hermitian
 * flavour, its first operator application D y.  Work is queued on `stream`; the call
 * returns once the set-up has finished.  On a stream other than the legacy default (NULL),
 * pseudo-Hermitian steps are captured into CUDA graphs (one per parity of the step index)
 * after their first eager run and replayed; results are bitwise those of eager launches
 * (LL_GRAPHS=0 in the environment keeps every launch eager).  LL_EINVAL on malformed input (unsorted spheres,
 * Miller indices that do not fit the grid, Q on the reciprocal lattice, a NaN or infinity in any
 * floating-point array, named in ll_last_error ...), checked on the host before any device work.
 * *out receives a handle to release with ll_destroy. */
int ll_create(const ll_system_desc* desc, void* stream, ll_handle** out);
int ll_destroy(ll_handle* h);

/* ll_create for another momentum transfer Q on the ground state of an existing chain `share`
 * (Sec. 2.1: Q = q + G may lie beyond the first Brillouin zone; Sec. 5 runs one recursion per
 * Q on one ground state).  The u_{vk}(r) grids, which depend on the ground state only (N^3 nks
 * nbnd complex values: 537 MB in FP32 on the 25 Ry, 8x8x8-k cell), are taken from `share`
 * instead of being built and stored again; everything that depends on Q (sphere(k+Q), u_kq,
 * beta_kq, the kinetic and Hartree tables, the vectors) is the new chain's own.  `desc` must
 * hold host arrays and the same ground state as `share`'s: precision, grid, k-points, bands,
 * sphere(k) and u_k (compared through a hash of those inputs; LL_EINVAL otherwise).  The
 * coefficients are those ll_create would give, bit for bit.  The grids stay allocated until the
 * last chain using them is destroyed; ll_bytes counts them in the chain that built them.
 * Waits for `share`'s stream once (its grids must be complete). */
int ll_create_sharing(const ll_system_desc* desc, ll_handle* share, void* stream, ll_handle** out);

/* Runs n_steps more Lanczos steps (Sec. 2.5), continuing from the resident state
 * (restart semantics of Sec. 3.2).  On return the arrays hold every coefficient so far
 * (`*steps_done` of them; capacity max_steps):
 *   alpha[i] = T_{i,i} = 0: every Lanczos vector has one non-zero half of the SBR pair and L
 *              maps one half to the other, so the diagonal of T vanishes in both recursions;
 *   beta[i]  = b_1 (i = 0) or T_{i+1,i};   gamma[i] (complex) = b_1 or T_{i,i+1};
 *   z[i] (complex) = z_{i+1} = ((y, 0), v_{i+1}) (Eq. 31).
 * Any of alpha, beta, gamma, z may be NULL.  LL_ENOTPD / LL_EBREAKDOWN stop the chain;
 * steps_done then counts the steps whose coefficients are valid.  A breakdown met only in
 * forming the coefficient after the n_steps asked for (the Krylov space exhausted at exactly
 * that length) returns LL_OK with every coefficient asked for; the chain stops, and the next
 * call returns LL_EBREAKDOWN. */
int ll_lanczos(ll_handle* h, int n_steps, double* alpha, double* beta, double* gamma, double* z, int* steps_done);

/* Spectrum of a handle's own coefficients on the device (Eqs. 32-33, 5):
 * chi(Q, w) = (4/Omega) b_1 sum_j z_j x_j with ((w + i eta) - T_M) x = e_1, using the first
 * m coefficients (m <= steps done; m <= 0: all).  eps_inv = 1 + 4 pi/|Q|^2 chi, eps = 1/eps_inv.
 * omega_ev [n_omega] and eta_ev in eV; chi, eps_inv, eps complex [n_omega] (host). */
int ll_lanczos_spectrum(ll_handle* h, int m, const double* omega_ev, int n_omega, double eta_ev,
                        double* chi, double* eps_inv, double* eps);

/* The same from caller-held coefficients (host arrays beta[m], gamma[m] complex, z[m]
 * complex), for a cell of volume omega_cell (bohr^3) and momentum q_cart (bohr^-1). */
int ll_spectrum(const double* beta, const double* gamma, const double* z, int m, double omega_cell,
                const double* q_cart, const double* omega_ev, int n_omega, double eta_ev, double* chi,
                double* eps_inv, double* eps, void* stream);

/* Extrapolation of the Lanczos coefficients (Sec. 2.5 end, Sec. 3.3, Appendix A): the
 * tridiagonal matrix of the m computed coefficients is continued to m_total x m_total at no
 * cost.  The off-diagonal coefficients of index i >= m (arrays as in ll_lanczos, index 0 being
 * b_1) take constant values: LL_EXTRAP_CONSTANT one value, the mean of beta (and of gamma)
 * over the indices max(1, m/2)..m-1; LL_EXTRAP_OSC (bi-constant) the means over the even and
 * over the odd indices of that range, each continuing its own parity.  z is continued with
 * zeros.  m >= 2 (>= 4 for LL_EXTRAP_OSC), m <= m_total <= LL_EXTRAP_MAX, else LL_EINVAL;
 * LL_EXTRAP_NO ignores m_total.  The means and the continued fraction run on the device. */
enum { LL_EXTRAP_NO = 0, LL_EXTRAP_CONSTANT = 1, LL_EXTRAP_OSC = 2 };
#define LL_EXTRAP_MAX 1000000

/* ll_lanczos_spectrum with the chain's first m coefficients (m <= 0: all) extrapolated to
 * m_total. */
int ll_lanczos_spectrum_x(ll_handle* h, int m, int kind, int m_total, const double* omega_ev, int n_omega,
                          double eta_ev, double* chi, double* eps_inv, double* eps);

/* ll_spectrum with the caller's m coefficients extrapolated to m_total. */
int ll_spectrum_x(const double* beta, const double* gamma, const double* z, int m, int kind, int m_total,
                  double omega_cell, const double* q_cart, const double* omega_ev, int n_omega, double eta_ev,
                  double* chi, double* eps_inv, double* eps, void* stream);

/* Allocation-free variant of ll_spectrum, for callers that cannot allocate device memory
 * while they run: services whose memory pool has already reserved the GPU's memory, and
 * latency-critical loops where a cudaMalloc/cudaFree (which may synchronise the device and
 * stall work on other streams) is not acceptable.  The paper has no counterpart; it is an
 * engineering addition.  Same arguments and results as ll_spectrum; the device staging of
 * the coefficients, the frequency grid and the three output arrays uses one static device
 * array compiled into the library (about 1.6 MB, held by every GPU that loads the library
 * until the process exits), so it accepts at most LL_SPECTRUM_STATIC_MAX_COEF coefficients
 * and LL_SPECTRUM_STATIC_MAX_OMEGA frequencies and returns LL_EINVAL with a message beyond
 * that.  It calls no device allocator.  The first call on a device looks up that device's
 * address of the array in the current context (make that first call before any stream
 * capture); the address is kept per device and looked up again when the device's context
 * has changed since (after a cudaDeviceReset, for instance).  Every call on a
 * device shares the one array and leaves its contents behind: calls whose work may overlap on
 * the GPU (other host threads, other streams) race and must be serialised by the caller.
 * Returns after the results are on the host. */
#define LL_SPECTRUM_STATIC_MAX_COEF 16384
#define LL_SPECTRUM_STATIC_MAX_OMEGA 16384
int ll_spectrum_static(const double* beta, const double* gamma, const double* z, int m, double omega_cell,
                       const double* q_cart, const double* omega_ev, int n_omega, double eta_ev, double* chi,
                       double* eps_inv, double* eps, void* stream);

/* One application of the SBR operator to a batch (Eqs. 24-28): out = (D + K) x when
 * upper != 0 (K omitted for IPA), out = D x otherwise, with D = P_c (H_{k+Q} - eps_{vk})
 * and the P_c of Eq. 16 on the output.  x and out are complex batches laid out per k as
 * [nbnd][npw_kq[k]] concatenated over k (host). */
int ll_apply(ll_handle* h, int upper, const double* x, double* out);

/* Bit-exact index map: for each k, each Miller of sphere(k+Q) -> its position in sphere(k)
 * or -1; int32 [sum npw_kq] concatenated (host). */
int ll_get_map(ll_handle* h, int* map_out);

/* The starting vector y = P_c u (Eq. 28) as a complex batch laid out like ll_apply's. */
int ll_get_start(ll_handle* h, double* y_out);

/* Kernel classes of the per-class device-time profile. */
enum {
  LL_PROF_ZINV = 0,     /* sphere -> columns, inverse FFT along axis 3 (the pseudo-Hermitian
                           vector update fused in front)                                 */
  LL_PROF_XY1 = 1,      /* per-plane 2D FFTs, V(r) x(r), response density                 */
  LL_PROF_HXC = 2,      /* Hartree + XC response potential of the density                 */
  LL_PROF_XY2 = 3,      /* per-plane forward 2D FFTs of v'(r) u(r)                         */
  LL_PROF_ZFWD = 4,     /* forward FFT along axis 3, columns -> sphere, fused with the
                           kinetic - eps, KB projector and P_c terms and the norm partials */
  LL_PROF_UPDATE = 5,   /* separate Lanczos update kernels (non-Hermitian), z reduction   */
  LL_NPROF = 6
};

/* Starts (enable != 0: counters cleared) or stops recording CUDA events around each
 * kernel class on the handle's stream.  Launch counting is always on. */
int ll_profile(ll_handle* h, int enable);

/* Device milliseconds per class summed over the recorded spans (ms[LL_NPROF]), kernel
 * launches per class (launches[LL_NPROF]) and in total since the last ll_profile(h, 1).
 * Synchronises the stream.  Any output may be NULL. */
int ll_profile_read(ll_handle* h, double* ms, long long* launches, long long* total);

/* Upper bound of the device bytes a handle for this descriptor will hold, the staging of a
 * spectrum excluded (input arrays are not read; computed on the host).  Returns LL_EINVAL when
 * the descriptor's sizes are missing. */
int ll_footprint(const ll_system_desc* desc, size_t* bytes);

/* Device bytes of the spectrum staging a handle adds for n_omega frequencies (the frequency
 * grid and the chi, eps^-1, eps outputs, plus the extrapolation constants). */
#define LL_SPECTRUM_BYTES(n_omega) ((size_t)(n_omega) * 56u + 256u)

/* f-sum printout (Sec. 2.1; the check of Sec. 3.3's post-processing): *moment = the trapezoid
 * integral over the grid of omega (-Im eps^-1(omega)) d omega (Ha^2; omega_ev in eV, eps_inv
 * complex interleaved, both host arrays of n_omega >= 2 points, increasing omega), computed on
 * the device in a fixed order; *expected (may be NULL) = (pi/2) omega_p^2 = (pi/2) 4 pi
 * nelec / omega_cell, which the moment approaches as the grid covers the spectrum (exactly
 * for a local potential; non-local projectors violate it slightly).  LL_EINVAL on bad sizes. */
int ll_fsum(const double* omega_ev, const double* eps_inv, int n_omega, double nelec, double omega_cell,
            double* moment, double* expected, void* stream);

/* Device bytes the handle holds now (every allocation, the spectrum staging included). */
int ll_bytes(ll_handle* h, size_t* bytes);

const char* ll_last_error(void);
const char* ll_version(void);

/* Measured FMA throughput of the current device in TFLOP/s (precision LL_PREC_FP32 or
 * LL_PREC_FP64): a kernel of independent FMA chains on every SM, the fastest of three timed
 * launches on `stream` (CUDA events).  The roofline denominator of the FFT kernels.  Allocates
 * and frees a small device buffer; returns after the measurement. */
int ll_fma_peak(int precision, double* tflops, void* stream);

/* ---- Request loop: continuous batching of chains (an engineering addition; the paper runs
 * one recursion per momentum transfer, Sec. 3.2).  A scheduler thread admits queued jobs in
 * arrival order while a slot is free and the job's device footprint fits the HBM budget, runs
 * every admitted chain on a stream of its own in rounds of `chunk` steps (their kernels
 * overlap on the GPU), and at a chain's last step evaluates its spectrum on the device and
 * frees its memory for the next admissions.  A job's results do not depend on the jobs
 * beside it. */
typedef struct ll_server ll_server;

enum { LL_JOB_QUEUED = 0, LL_JOB_RUNNING = 1, LL_JOB_DONE = 2, LL_JOB_FAILED = 3 };

typedef struct {
  ll_system_desc sys;       /* copied at submit; sys.max_steps >= n_steps                   */
  int n_steps;              /* Lanczos steps of the job                                    */
  const double* omega_ev;   /* [n_omega] spectrum grid (eV); n_omega = 0: coefficients only */
  int n_omega;
  double eta_ev;            /* broadening (eV)                                             */
} ll_job_desc;

typedef struct {
  int status;               /* LL_OK, or the error that ended the job                      */
  int steps_done;
  double queue_s, run_s;    /* seconds waiting for admission; from admission to the end    */
  double* beta;             /* optional caller buffers, filled once the job has ended:     */
  double* gamma;            /*   beta [n_steps]; gamma, z complex [n_steps]                */
  double* z;
  double* chi;              /*   chi, eps_inv, eps complex [n_omega]                       */
  double* eps_inv;
  double* eps;
} ll_job_result;

/* hbm_budget_bytes caps the summed device footprint of running chains; max_slots caps their
 * number.  The scheduler thread uses the device current at this call. */
int ll_server_create(size_t hbm_budget_bytes, int max_slots, ll_server** out);
/* Steps queued per chain per round (default 64). */
int ll_server_set_chunk(ll_server* s, int steps);
/* Copies the job; LL_ENOMEM when its footprint exceeds the whole budget, LL_EINVAL when the
 * descriptor is malformed: a missing array, an empty sphere, a NaN or an infinity in any
 * floating-point input (further checks happen at admission and end the job FAILED). */
int ll_submit(ll_server* s, const ll_job_desc* job, uint64_t* job_id);
/* *state = LL_JOB_*; when res is given, fills it (results once the job has ended). */
int ll_poll(ll_server* s, uint64_t job_id, int* state, ll_job_result* res);
/* Cancels a job.  A queued job leaves the queue at once.  A running chain stops at the end of
 * the scheduler's current round, when none of its kernels is in flight; it keeps the
 * coefficients (and the spectrum, when a grid was given) of the steps it finished, and its
 * memory goes back to the budget.  Either way the job ends FAILED with status LL_ECANCELED.
 * A job that reaches its last step in that round, or that has already ended, keeps its
 * outcome (LL_OK).  LL_ENOTFOUND for an unknown id. */
int ll_cancel(ll_server* s, uint64_t job_id);
/* Frees the record of a job that has ended (after its results were polled); its id is unknown
 * from then on.  LL_PENDING while the job is queued or running, LL_ENOTFOUND for an unknown id.
 * Without it a server keeps every ended job's results until ll_server_destroy. */
int ll_release(ll_server* s, uint64_t job_id);
/* Device bytes held by running chains now and at most so far; running and queued jobs. */
int ll_server_stats(ll_server* s, size_t* used, size_t* peak, int* running, int* queued);
const char* ll_server_last_error(void);
/* Stops the scheduler after its current round; queued jobs end FAILED. */
int ll_server_destroy(ll_server* s);

#ifdef __cplusplus
}
#endif
#endif
