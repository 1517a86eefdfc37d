// Host side of libswkb.so: plan construction (mode set, ray layout, medium
// tables, device buffers), the screen loop, and the C ABI of include/swkb.h.
//
// Everything the device path needs in FP64 is prepared here:
//   - the medium table as per-interval quintic coefficients of eps - eps_ref
//     (quintic Hermite in z from eps, eps_z, eps_zz; reading of the paper's
//     silent medium representation), cast to FP32 for the mixed path;
//   - the per-screen RK4 stage columns (linear in x, right limit at the start
//     of a screen and left limit at its end);
//   - the mode table kappa_n = 2 pi n / (k L) (Eq. fourier_psi with the
//     origin at the bottom of the period), P_bar_n = sqrt(eps_ref - kappa_n^2)
//     and the range-phase carry exp(i k dx P_bar_n) (reduced mod 2 pi in FP64);
//   - DFT twiddles and the top absorber window.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "swkb.h"
#include "swkb_internal.h"

using namespace swkb;

namespace {
// NVTX range for profilers (ncu --nvtx, nsys); a no-op without one attached
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

thread_local std::string g_err;

swkb_status fail(swkb_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CK(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(SWKB_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                      \
  } while (0)

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(long long v) {
  int l = 0;
  while ((1LL << l) < v) ++l;
  return l;
}

}  // namespace

void swkb::set_last_error(const char* msg) { g_err = msg ? msg : ""; }

struct swkb_plan {
  // problem
  int precision = SWKB_FP64;
  int bc = SWKB_BC_PERIODIC;
  int mirror = 0;  // 0 periodic, +1 Neumann, -1 Dirichlet
  int sym = 0;     // grounded: march modes n >= 0 only, sum the physical half only
  int Mr = 0;      // marched modes
  int n_tiles_run = 0;
  int n_z = 0, N = 0, N1 = 1, N2 = 1, log2N2 = 0;
  int n_max = 0, M = 0, R = 1, N_r = 0, G = 0, NRT = 0, Nt = 0;
  double k = 0, z_a = 0, z_b = 0, x0 = 0, dx = 0, L = 0, dz = 0, z_lo = 0;
  double eps_ref = 0, absorber_frac = 0;
  // resummation tiling
  int PW = 8, TM = 256, n_tiles = 0, n_groups = 1, modes_per_group = 1, wcap = 0;
  int ctas_per_sm = 6, sms = 1;
  int alloc_groups = 0, alloc_tiles = 0;   // buffer sizes: max over tuning candidates
  // medium
  int n_cols = 0, n_p = 0, n_int = 0;
  int pieces = 0;   // FP32: cubic pieces per table interval (0: the quintic)
  double z0p = 0, dzp = 0;
  std::vector<double> x_cols;
  int stage_rows = 1;  // screens q >= stage_rows - 1 share the last row
  bool autotune = false;
  bool reuse_rays = false;   // one table column and opted in: march once per call
  bool rays_ready = false;   // (within the current enqueue sequence)
  std::vector<double> pbar;  // host copy of P_bar_n (FP64)
  std::vector<double> ephi;  // exp(i k dx P_bar_n), interleaved
  // device
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* coef = nullptr;
  void* tw = nullptr;
  void* W = nullptr;
  void* kappa = nullptr;
  void* pbar_d = nullptr;
  void* pbar2_d = nullptr;
  void* ephi_d = nullptr;
  void* u = nullptr;
  void* part = nullptr;
  void* Y = nullptr;
  void* c = nullptr;
  void* cpol = nullptr;   // FP32: (|c_n|, arg(c_n) / 2 pi) of c
  void* rd = nullptr;
  void* rph = nullptr;
  void* ra = nullptr;
  // fields between screens: ray data of planes - 1 inner planes, the mode
  // coefficients of one plane, its range-phase factors
  int planes = 0;
  void* pl_d = nullptr;
  void* pl_ph = nullptr;
  void* pl_a = nullptr;
  void* c_plane = nullptr;
  void* cpol_plane = nullptr;
  void* ephi_pl = nullptr;
  int* jlo = nullptr;
  int* jlo_neg = nullptr;
  unsigned* status = nullptr;
  int* stage_c = nullptr;
  void* stage_th = nullptr;
  double* io = nullptr;  // complex128 staging, max(N, n_z) values
  size_t bytes = 0;
  int alloc_calls = 0;   // device allocations attempted (fault injection counts them)
  std::vector<void*> allocs;
  // accounting
  swkb_plan_stats stats{};
  unsigned timing = 0;               // bit k: time kernel kind k with CUDA events
  int timing_every = 1;              // time one launch in timing_every per kind
  bool timing_serial = false;        // while timing: march on the plan stream too
  uint64_t timing_seen[SWKB_KERNEL_KINDS] = {};
  std::vector<cudaEvent_t> events;   // pool, reused every run
  struct Mark { int kind; int e0, e1; };
  std::vector<Mark> marks;           // pending, harvested after a sync
  // captured propagations, replayed with cudaGraphLaunch
  struct Graph {
    int q0, n, snap, timing, every;
    const double* in;
    double* out;
    cudaGraphExec_t exec;
    std::vector<Mark> marks;         // event pairs the graph records
    swkb_plan_stats delta;           // launches / screens one replay adds
  };
  std::vector<Graph> graphs;
  bool use_graphs = true;
  bool fuse_reduce = true;   // DFT pass 1 forms the field from the partials
  // rays on a second stream: a second set of ray and bracket buffers, the
  // stream, and per set an event "rays ready" and "set free again"
  bool overlap = false;
  cudaStream_t ray_stream = nullptr;
  cudaEvent_t ev_rays[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  void* rd1 = nullptr;
  void* rph1 = nullptr;
  void* ra1 = nullptr;
  int* jlo1 = nullptr;
  int* jlo_neg1 = nullptr;
  // patch-wise Fourier continuation (SWKB_BC_OPEN): patches of fc_pat grid
  // points every fc_stride points, fc_P of them, each continued to fc_Np
  bool fc = false;
  int fc_pat = 0, fc_ov = 0, fc_stride = 0, fc_P = 0, fc_Np = 0;
  void* fc_cont = nullptr;    // [FC_C][FC_D] continuation operator, FP64
  void* fc_tw = nullptr;      // [Np] exp(-2 pi i k / Np), FP64
  void* fc_cf = nullptr;      // [P][M] mode coefficients of every patch
  void* fc_cf_plane = nullptr;  // [P][M] the same carried to a plane inside the screen
  int* fc_win_p = nullptr;    // [NRT] first patch weighting launch point j
  void* fc_win_s = nullptr;   // [NRT] (S^{p0}, S^{p0+1}) at launch point j
};

namespace {

// Fault injection for tests, on the host: SWKB_FAIL_ALLOC_AT=n makes the n-th
// device allocation of a plan (counted from 1) fail as if the device were out
// of memory, without calling cudaMalloc.
swkb_status dev_alloc(swkb_plan* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  ++p->alloc_calls;
  if (const char* fa = getenv("SWKB_FAIL_ALLOC_AT")) {
    if (atoi(fa) == p->alloc_calls)
      return fail(SWKB_ERR_OOM, "device allocation %d refused (SWKB_FAIL_ALLOC_AT)", p->alloc_calls);
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SWKB_ERR_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  p->allocs.push_back(*ptr);
  p->bytes += bytes;
  return SWKB_OK;
}

#define TRY(x)                      \
  do {                              \
    swkb_status s_ = (x);           \
    if (s_ != SWKB_OK) return s_;   \
  } while (0)

// Columns (c, c + 1) and weight th of column c + 1 at range x.  right: take
// the right limit at a column position (x_cols[c] <= x), else the left one.
void column_weights(const std::vector<double>& xc, double x, bool right, int* c, double* th) {
  const int n = (int)xc.size();
  if (n == 1) { *c = 0; *th = 0.0; return; }
  int cnt = 0;
  for (int i = 0; i < n; ++i) cnt += right ? (xc[i] <= x) : (xc[i] < x);
  int cc = std::min(std::max(cnt - 1, 0), n - 2);
  const double span = xc[cc + 1] - xc[cc];
  double t = span <= 0 ? 0.0 : (x - xc[cc]) / span;
  *c = cc;
  *th = std::min(std::max(t, 0.0), 1.0);
}

template <typename T>
swkb_status upload(swkb_plan* p, void** dst, const std::vector<double>& v) {
  std::vector<T> tmp(v.begin(), v.end());
  TRY(dev_alloc(p, dst, tmp.size() * sizeof(T)));
  CK(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SWKB_OK;
}

}  // namespace

swkb_status swkb::status_from_bits(unsigned bits) {
  if (bits & ST_BOUNDS)
    return fail(SWKB_ERR_CUDA, "a device index left its buffer (bounds-checked build)");
  // a turning point comes first: the FP32 march carries a ray that met one
  // on with NaN values, whose landings then also fail the order check
  if (bits & ST_TURNING) return fail(SWKB_ERR_TURNING, "turning point on a ray (eps - Q^2 <= 0)");
  if (bits & ST_CAUSTIC)
    return fail(SWKB_ERR_CAUSTIC,
                "caustic between screens (Z_s <= 0 or ray landings out of order); "
                "use a smaller screen spacing");
  if (bits & ST_RANGE) return fail(SWKB_ERR_RANGE, "a ray left the permittivity table");
  if (bits & ST_COVER) return fail(SWKB_ERR_RANGE, "ghost rays do not cover the screen");
  return SWKB_OK;
}

namespace {

// Intervals of the FP32 medium table of one column (layout in swkb_internal.h).
int table32_intervals(const swkb_plan* p) { return (p->mirror ? 2 : 1) * p->n_int + 1; }

// Quintic Hermite interpolant of eps - eps_ref on every profile interval, as
// monomial coefficients a0..a5 in t in [0, 1] (8 slots per interval).
std::vector<double> quintic_coefficients(const swkb_plan* p, const swkb_profile* prof) {
  std::vector<double> coef((size_t)p->n_cols * p->n_int * 8, 0.0);
  const double h = p->dzp;
  for (int c = 0; c < p->n_cols; ++c) {
    const double* e = prof->eps + (size_t)c * p->n_p;
    const double* ez = prof->eps_z + (size_t)c * p->n_p;
    const double* ezz = prof->eps_zz + (size_t)c * p->n_p;
    for (int i = 0; i < p->n_int; ++i) {
      const double f0 = e[i] - p->eps_ref, f1 = e[i + 1] - p->eps_ref;
      const double a0 = f0, a1 = h * ez[i], a2 = 0.5 * h * h * ezz[i];
      const double A = f1 - a0 - a1 - a2;
      const double B = h * ez[i + 1] - a1 - 2.0 * a2;
      const double C = h * h * ezz[i + 1] - 2.0 * a2;
      double* o = coef.data() + ((size_t)c * p->n_int + i) * 8;
      o[0] = a0; o[1] = a1; o[2] = a2;
      o[3] = 10.0 * A - 4.0 * B + 0.5 * C;
      o[4] = -15.0 * A + 7.0 * B - C;
      o[5] = 6.0 * A - 3.0 * B + 0.5 * C;
    }
  }
  return coef;
}

// value, first and second t-derivative of a quintic at t
void quintic_eval(const double* a, double t, double& v, double& d1, double& d2) {
  v = ((((a[5] * t + a[4]) * t + a[3]) * t + a[2]) * t + a[1]) * t + a[0];
  d1 = (((5.0 * a[5] * t + 4.0 * a[4]) * t + 3.0 * a[3]) * t + 2.0 * a[2]) * t + a[1];
  d2 = ((20.0 * a[5] * t + 12.0 * a[4]) * t + 6.0 * a[3]) * t + 2.0 * a[2];
}

// Cubic Hermite piece s of S of a quintic (value and slope matched at both
// ends), as monomial coefficients b0..b3 in tau in [0, 1].
void cubic_piece(const double* a, int s, int S, double* b) {
  double f0, d0, g0, f1, d1, g1;
  quintic_eval(a, (double)s / S, f0, d0, g0);
  quintic_eval(a, (double)(s + 1) / S, f1, d1, g1);
  d0 /= S; d1 /= S;                                  // d/dtau = (1/S) d/dt
  b[0] = f0;
  b[1] = d0;
  b[2] = 3.0 * (f1 - f0) - 2.0 * d0 - d1;
  b[3] = 2.0 * (f0 - f1) + d0 + d1;
}

// FP32 plans evaluate each interval's quintic through S cubic Hermite pieces
// (6 FMAs per lookup instead of 12).  S is the smallest of 1, 2, 4, 8, 16 for
// which, at the quarter points of every piece, value, slope and curvature of
// the pieces stay within 1e-7, 1e-6 and 1e-4 of the table's largest |e|, |e_z|
// and |e_zz| (e = eps - eps_ref): far below what the FP32 march resolves.
// 0 when none does (the quintic itself is evaluated).
int choose_pieces(const swkb_plan* p, const std::vector<double>& coef) {
  const double h = p->dzp;
  const size_t n = (size_t)p->n_cols * p->n_int;
  double E0 = 0, E1 = 0, E2 = 0;
  for (size_t i = 0; i < n; ++i) {
    const double* a = coef.data() + i * 8;
    for (double t : {0.0, 1.0}) {
      double v, d1, d2;
      quintic_eval(a, t, v, d1, d2);
      E0 = std::max(E0, fabs(v));
      E1 = std::max(E1, fabs(d1) / h);
      E2 = std::max(E2, fabs(d2) / (h * h));
    }
  }
  const double tol[3] = {1e-7 * E0, 1e-6 * E1, 1e-4 * E2};
  // largest deviations of S pieces from the quintic (value, slope, curvature);
  // with stop set, returns as soon as one exceeds its bound
  auto worst = [&](int S, double dev[3], bool stop) {
    dev[0] = dev[1] = dev[2] = 0.0;
    for (size_t i = 0; i < n; ++i) {
      const double* a = coef.data() + i * 8;
      for (int s = 0; s < S; ++s) {
        double b[4];
        cubic_piece(a, s, S, b);
        for (double tau : {0.25, 0.5, 0.75}) {
          double v, d1, d2;
          quintic_eval(a, (s + tau) / S, v, d1, d2);
          const double cv = ((b[3] * tau + b[2]) * tau + b[1]) * tau + b[0];
          const double c1 = ((3.0 * b[3] * tau + 2.0 * b[2]) * tau + b[1]) * S;
          const double c2 = (6.0 * b[3] * tau + 2.0 * b[2]) * S * S;
          dev[0] = std::max(dev[0], fabs(cv - v));
          dev[1] = std::max(dev[1], fabs(c1 - d1) / h);
          dev[2] = std::max(dev[2], fabs(c2 - d2) / (h * h));
          if (stop && (dev[0] > tol[0] || dev[1] > tol[1] || dev[2] > tol[2])) return false;
        }
      }
    }
    return dev[0] <= tol[0] && dev[1] <= tol[1] && dev[2] <= tol[2];
  };
  double dev[3];
  if (worst(1, dev, false)) return 1;
  // cubic Hermite errors fall as S^-4 (value), S^-3 (slope), S^-2 (curvature):
  // start from the S the single-piece deviations predict, then verify
  auto ratio = [](double d, double t) { return t > 0 ? d / t : (d > 0 ? 1e300 : 0.0); };
  const double need = std::max({pow(ratio(dev[0], tol[0]), 0.25), pow(ratio(dev[1], tol[1]), 1.0 / 3.0),
                                sqrt(ratio(dev[2], tol[2]))});
  const long long ext = (long long)(p->mirror ? 2 : 1) * p->n_int;
  int S = 2;
  while (S < need && S < 16) S *= 2;
  for (; S <= 16; S *= 2) {
    if (ext * S >= (1LL << 22)) break;            // FP32 positions stay exact below 2^22
    if (worst(S, dev, true)) return S;
  }
  return 0;
}

// choose_pieces depends only on the table (and eps_ref, the ground
// reflection): remembered by a 64-bit FNV-1a hash of those, so that the
// budget estimate and the creation of the same request's plan scan it once.
uint64_t table_hash(const swkb_plan* p, const swkb_profile* prof) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* data, size_t bytes) {
    const unsigned char* c = (const unsigned char*)data;
    for (size_t i = 0; i < bytes; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  };
  const size_t nt = (size_t)p->n_cols * p->n_p;
  mix(prof->eps, nt * sizeof(double));
  mix(prof->eps_z, nt * sizeof(double));
  mix(prof->eps_zz, nt * sizeof(double));
  const double sc[2] = {p->eps_ref, p->dzp};
  const int ic[3] = {p->n_cols, p->n_p, p->mirror};
  mix(sc, sizeof(sc));
  mix(ic, sizeof(ic));
  return h;
}

std::mutex g_pieces_mutex;
std::map<uint64_t, int> g_pieces_cache;

int pieces_for(const swkb_plan* p, const swkb_profile* prof) {
  const uint64_t key = table_hash(p, prof);
  {
    std::lock_guard<std::mutex> lk(g_pieces_mutex);
    auto it = g_pieces_cache.find(key);
    if (it != g_pieces_cache.end()) return it->second;
  }
  const int S = choose_pieces(p, quintic_coefficients(p, prof));
  std::lock_guard<std::mutex> lk(g_pieces_mutex);
  if (g_pieces_cache.size() >= 256) g_pieces_cache.clear();
  g_pieces_cache[key] = S;
  return S;
}

// C-infinity step of the partition of unity: e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}),
// 0 for t <= 0, 1 for t >= 1.
double fc_step(double t) {
  if (t <= 0.0) return 0.0;
  if (t >= 1.0) return 1.0;
  const double a = exp(-1.0 / t), b = exp(-1.0 / (1.0 - t));
  return a / (a + b);
}

// Weight of patch pt at grid-unit position u: rising over the patch's first
// fc_ov points, falling over its last fc_ov, zero outside it.
double fc_weight(const swkb_plan* p, int pt, double u) {
  const double s = (double)pt * p->fc_stride, e = s + p->fc_pat - 1, w = p->fc_ov - 1;
  return fc_step((u - s) / w) * (1.0 - fc_step((u - (e - w)) / w));
}

// Continuation operator, patch twiddles, per-launch-point patch weights and
// the per-patch coefficient buffer of a patch-wise plan.
template <typename T>
swkb_status build_fc(swkb_plan* p) {
  using V = typename C2<T>::type;
  {
    const double* op = fc_continuation_host();
    std::vector<double> cont(op, op + FC_CONT_ROWS * FC_CONT_COLS);
    TRY(upload<double>(p, &p->fc_cont, cont));
  }
  {
    std::vector<double> tw(2 * (size_t)p->fc_Np);
    for (int k = 0; k < p->fc_Np; ++k) {
      const double a = 2.0 * M_PI * ((double)k / p->fc_Np);
      tw[2 * k] = cos(a);
      tw[2 * k + 1] = -sin(a);
    }
    TRY(upload<double>(p, &p->fc_tw, tw));
  }
  {
    // launch point j sits at grid position (j - G) R; at most two patches
    // weight it: the first with a non-zero weight and the next one
    std::vector<int> wp(p->NRT, 0);
    std::vector<double> ws(2 * (size_t)p->NRT, 0.0);
    for (int j = 0; j < p->NRT; ++j) {
      const double u = (double)(j - p->G) * p->R;
      int first = -1;
      for (int pt = std::max(0, (int)floor((u - p->fc_pat + 1) / p->fc_stride));
           pt < p->fc_P && pt * (double)p->fc_stride <= u; ++pt)
        if (fc_weight(p, pt, u) > 0.0) { first = pt; break; }
      if (first < 0) continue;
      wp[j] = first;
      ws[2 * (size_t)j] = fc_weight(p, first, u);
      ws[2 * (size_t)j + 1] = first + 1 < p->fc_P ? fc_weight(p, first + 1, u) : 0.0;
    }
    TRY(dev_alloc(p, (void**)&p->fc_win_p, wp.size() * sizeof(int)));
    CK(cudaMemcpy(p->fc_win_p, wp.data(), wp.size() * sizeof(int), cudaMemcpyHostToDevice));
    TRY(upload<T>(p, &p->fc_win_s, ws));
  }
  TRY(dev_alloc(p, &p->fc_cf, (size_t)p->fc_P * p->M * sizeof(V)));
  if (p->planes > 1) TRY(dev_alloc(p, &p->fc_cf_plane, (size_t)p->fc_P * p->M * sizeof(V)));
  return SWKB_OK;
}

template <typename T>
swkb_status build_device(swkb_plan* p, const swkb_profile* prof) {
  using V = typename C2<T>::type;
  const int M = p->M, N = p->N;
  // medium coefficient table (eps - eps_ref), 8 slots per interval
  {
    const std::vector<double> coef = quintic_coefficients(p, prof);
    if (sizeof(T) == 8) {
      TRY(upload<T>(p, &p->coef, coef));
    } else {
      // FP32 layout: reflected intervals below z_a (grounded), the profile's
      // intervals, one continuation interval.  A reflected interval holds
      // p(1 - t) and the continuation p_last(1 + t), re-expanded in t.
      const int lo = p->mirror ? p->n_int : 0, nt = table32_intervals(p);
      std::vector<double> c32((size_t)p->n_cols * nt * 8, 0.0);
      static const double binom[6][6] = {{1, 0, 0, 0, 0, 0}, {1, 1, 0, 0, 0, 0},
                                         {1, 2, 1, 0, 0, 0}, {1, 3, 3, 1, 0, 0},
                                         {1, 4, 6, 4, 1, 0}, {1, 5, 10, 10, 5, 1}};
      for (int c = 0; c < p->n_cols; ++c)
        for (int k = 0; k < nt; ++k) {
          const int i = k < lo ? lo - 1 - k : std::min(k - lo, p->n_int - 1);
          const double sgn = k < lo ? -1.0 : 1.0;        // t -> 1 - t or t -> 1 + t
          const bool shift = k < lo || k - lo >= p->n_int;
          const double* a = coef.data() + ((size_t)c * p->n_int + i) * 8;
          double* o = c32.data() + ((size_t)c * nt + k) * 8;
          if (!shift) {
            for (int j = 0; j < 6; ++j) o[j] = a[j];
          } else {
            // sum_m a_m (1 + sgn t)^m = sum_j t^j sgn^j sum_{m >= j} C(m, j) a_m
            for (int j = 0; j < 6; ++j) {
              double acc = 0;
              for (int m = 5; m >= j; --m) acc += binom[m][j] * a[m];
              o[j] = (j & 1) ? sgn * acc : acc;
            }
          }
        }
      if (p->pieces > 0) {
        // cubic pieces, 4 floats each, S per extended interval
        const int S = p->pieces;
        std::vector<double> cub((size_t)p->n_cols * nt * S * 4);
        for (size_t k = 0; k < (size_t)p->n_cols * nt; ++k)
          for (int sp = 0; sp < S; ++sp) cubic_piece(c32.data() + k * 8, sp, S, &cub[(k * S + sp) * 4]);
        TRY(upload<T>(p, &p->coef, cub));
      } else {
        TRY(upload<T>(p, &p->coef, c32));
      }
    }
  }
  // RK4 stage columns for screens 0 .. stage_rows - 1
  {
    const int S = 2 * p->Nt + 1;
    std::vector<int> sc((size_t)p->stage_rows * S);
    std::vector<double> st((size_t)p->stage_rows * S);
    const double h = p->dx / p->Nt;
    for (int q = 0; q < p->stage_rows; ++q) {
      const double xq = p->x0 + q * p->dx;
      const double xn = p->x0 + (q + 1) * p->dx;
      for (int l = 0; l < S; ++l) {
        const bool last = (l == S - 1);
        const double x = last ? xn : xq + 0.5 * l * h;
        int c;
        double th;
        column_weights(p->x_cols, x, !last, &c, &th);
        sc[(size_t)q * S + l] = c;
        st[(size_t)q * S + l] = th;
      }
    }
    TRY(dev_alloc(p, (void**)&p->stage_c, sc.size() * sizeof(int)));
    CK(cudaMemcpy(p->stage_c, sc.data(), sc.size() * sizeof(int), cudaMemcpyHostToDevice));
    TRY(upload<T>(p, &p->stage_th, st));
  }
  // modes
  {
    std::vector<double> kap(M), pb(M), pb2(M);
    p->pbar.assign(M, 0.0);
    p->ephi.assign(2 * (size_t)M, 0.0);
    for (int i = 0; i < M; ++i) {
      const int n = i - p->n_max;
      kap[i] = 2.0 * M_PI * n / (p->k * p->L);
      pb2[i] = p->eps_ref - kap[i] * kap[i];
      pb[i] = sqrt(pb2[i]);
      p->pbar[i] = pb[i];
      const double phi = fmod(p->k * p->dx * pb[i], 2.0 * M_PI);
      p->ephi[2 * i] = cos(phi);
      p->ephi[2 * i + 1] = sin(phi);
    }
    TRY(upload<T>(p, &p->kappa, kap));
    TRY(upload<T>(p, &p->pbar_d, pb));
    TRY(upload<T>(p, &p->pbar2_d, pb2));
    TRY(upload<T>(p, &p->ephi_d, p->ephi));
  }
  if (p->fc) TRY(build_fc<T>(p));
  // twiddles exp(-2 pi i k / N)
  if (!p->fc) {
    std::vector<double> tw(2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
      const double a = 2.0 * M_PI * ((double)k / N);
      tw[2 * k] = cos(a);
      tw[2 * k + 1] = -sin(a);
    }
    TRY(upload<T>(p, &p->tw, tw));
  }
  // absorber
  if (p->absorber_frac > 0) {
    std::vector<double> w(N, 1.0);
    const double H = p->z_b - p->z_a, f = p->absorber_frac;
    for (int m = 0; m < N; ++m) {
      const double z = p->z_lo + p->dz * m;
      const double d = p->mirror ? fabs(z - p->z_a) : (z - p->z_a);
      if (d > (1.0 - f) * H) {
        const double cth = cos(0.5 * M_PI * (d - (1.0 - f) * H) / (f * H));
        w[m] = cth * cth;
      }
    }
    TRY(upload<T>(p, &p->W, w));
  }
  // work buffers
  TRY(dev_alloc(p, &p->u, (size_t)N * sizeof(V)));
  TRY(dev_alloc(p, &p->part, (size_t)p->alloc_groups * N * sizeof(V)));
  if (!p->fc) TRY(dev_alloc(p, &p->Y, (size_t)N * sizeof(V)));
  TRY(dev_alloc(p, &p->c, (size_t)M * sizeof(V)));
  if (sizeof(T) == 4) TRY(dev_alloc(p, &p->cpol, (size_t)M * sizeof(V)));
  const size_t rays = (size_t)p->NRT * p->Mr;
  TRY(dev_alloc(p, &p->rd, rays * sizeof(T)));
  TRY(dev_alloc(p, &p->rph, rays * sizeof(T)));
  TRY(dev_alloc(p, &p->ra, rays * sizeof(T)));
  if (p->planes > 1) {
    const size_t pr = (size_t)(p->planes - 1) * rays;
    TRY(dev_alloc(p, &p->pl_d, pr * sizeof(T)));
    TRY(dev_alloc(p, &p->pl_ph, pr * sizeof(T)));
    TRY(dev_alloc(p, &p->pl_a, pr * sizeof(T)));
    TRY(dev_alloc(p, &p->c_plane, (size_t)M * sizeof(V)));
    if (sizeof(T) == 4) TRY(dev_alloc(p, &p->cpol_plane, (size_t)M * sizeof(V)));
    TRY(dev_alloc(p, &p->ephi_pl, (size_t)(p->planes - 1) * M * sizeof(V)));
  }
  const size_t jn = (size_t)(p->alloc_tiles + 1) * p->Mr;
  TRY(dev_alloc(p, (void**)&p->jlo, jn * sizeof(int)));
  CK(cudaMemsetAsync(p->jlo, 0, jn * sizeof(int), p->stream));
  if (p->sym) {
    TRY(dev_alloc(p, (void**)&p->jlo_neg, jn * sizeof(int)));
    CK(cudaMemsetAsync(p->jlo_neg, 0, jn * sizeof(int), p->stream));
  }
  if (p->overlap) {
    TRY(dev_alloc(p, &p->rd1, rays * sizeof(T)));
    TRY(dev_alloc(p, &p->rph1, rays * sizeof(T)));
    TRY(dev_alloc(p, &p->ra1, rays * sizeof(T)));
    TRY(dev_alloc(p, (void**)&p->jlo1, jn * sizeof(int)));
    CK(cudaMemsetAsync(p->jlo1, 0, jn * sizeof(int), p->stream));
    if (p->sym) {
      TRY(dev_alloc(p, (void**)&p->jlo_neg1, jn * sizeof(int)));
      CK(cudaMemsetAsync(p->jlo_neg1, 0, jn * sizeof(int), p->stream));
    }
  }
  TRY(dev_alloc(p, (void**)&p->status, sizeof(unsigned)));
  CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), p->stream));
  TRY(dev_alloc(p, (void**)&p->io, 2 * (size_t)std::max(N, p->n_z) * sizeof(double)));
  if (p->fc)
    CK(prepare_fc_kernels<T>((int)fc_resum_smem_bytes<T>(p->wcap, p->TM),
                             (int)fc_modes_smem_bytes<T>(p->fc_Np)));
  else
    CK(prepare_kernels<T>((int)resum_smem_bytes<T>(p->wcap, p->TM)));
  return SWKB_OK;
}

// ---------------------------------------------------------------------------
// per-kernel accounting: launch counts always, CUDA-event timing on request
// ---------------------------------------------------------------------------
swkb_status event_at(swkb_plan* p, int idx) {
  while ((int)p->events.size() <= idx) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    p->events.push_back(e);
  }
  return SWKB_OK;
}

// propagate calls run the march on the ray stream unless the plan has none or
// serial timing is on
bool overlapped(const swkb_plan* p) { return p->overlap && !p->timing_serial; }

int timing_key(const swkb_plan* p) { return (int)p->timing | (p->timing_serial ? SWKB_TIME_SERIAL : 0); }

template <typename F>
swkb_status timed_on(swkb_plan* p, cudaStream_t stream, int kind, int n_launches, F&& launch) {
  int e0 = -1, e1 = -1;
  const bool on = ((p->timing >> kind) & 1u) && (p->timing_seen[kind]++ % p->timing_every == 0);
  if (on) {
    e0 = 2 * (int)p->marks.size();
    e1 = e0 + 1;
    TRY(event_at(p, e1));
    // "external" records become event-record nodes when the stream is being
    // captured into a graph (and are plain records otherwise)
    CK(cudaEventRecordWithFlags(p->events[e0], stream, cudaEventRecordExternal));
  }
  CK(launch());
  if (on) {
    CK(cudaEventRecordWithFlags(p->events[e1], stream, cudaEventRecordExternal));
    p->marks.push_back({kind, e0, e1});
    p->stats.kernel_timed[kind] += n_launches;
  }
  p->stats.launches += n_launches;
  p->stats.kernel_launches[kind] += n_launches;
  return SWKB_OK;
}

template <typename F>
swkb_status timed(swkb_plan* p, int kind, int n_launches, F&& launch) {
  return timed_on(p, p->stream, kind, n_launches, launch);
}

// after the stream has been synchronised
swkb_status harvest(swkb_plan* p) {
  for (const auto& m : p->marks) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p->events[m.e0], p->events[m.e1]));
    p->stats.kernel_ms[m.kind] += ms;
  }
  p->marks.clear();
  return SWKB_OK;
}

// ---------------------------------------------------------------------------
// kernel argument builders
// ---------------------------------------------------------------------------
template <typename T>
MarchArgs<T> march_args(const swkb_plan* p, int q) {
  MarchArgs<T> a;
  a.med.coef = (const T*)p->coef;
  a.med.n_int = p->n_int;
  a.med.col_stride = (long long)p->n_int * 8;
  a.med.z0 = (T)p->z0p;
  a.med.inv_h = (T)(1.0 / p->dzp);
  a.med.inv_h2 = (T)(2.0 / (p->dzp * p->dzp));
  a.med.mirrored = p->mirror != 0;
  a.med.z_mirror = (T)p->z_a;
  a.med.top = (T)p->n_int;
  a.med.pieces = 0;
  a.med.size = (long long)p->n_cols * p->n_int * 8;
  if (sizeof(T) == 4) {
    // reflection stored in the table; positions in table intervals
    const double z0 = p->mirror ? p->z0p - p->n_int * p->dzp : p->z0p;
    // with cubic pieces, positions and derivatives are in piece units
    const int S = p->pieces > 0 ? p->pieces : 1;
    const double hs = p->dzp / S;
    a.med.n_int = (p->mirror ? 2 : 1) * p->n_int * S;
    a.med.col_stride = (long long)table32_intervals(p) * (p->pieces > 0 ? 4 * S : 8);
    a.med.z0 = (T)z0;
    a.med.inv_h = (T)(1.0 / hs);
    a.med.inv_h2 = (T)(2.0 / (hs * hs));
    a.med.mirrored = 0;
    a.med.pieces = p->pieces;
    a.med.size = (long long)p->n_cols * a.med.col_stride;
    a.med.top = (T)a.med.n_int;
    a.u_lo = (T)((p->z_lo - z0) / hs);
    a.u_dz = (T)(p->dz / hs);
  } else {
    a.u_lo = a.u_dz = T(0);
  }
  const int S = 2 * p->Nt + 1;
  const int row = std::min(std::max(q, 0), p->stage_rows - 1);
  a.st.c = p->stage_c + (size_t)row * S;
  a.st.th = (const T*)p->stage_th + (size_t)row * S;
  a.kappa = (const T*)p->kappa;
  a.pbar = (const T*)p->pbar_d;
  a.pbar2 = (const T*)p->pbar2_d;
  a.Mr = p->Mr; a.mode_off = p->sym ? p->n_max : 0;
  a.NRT = p->NRT; a.G = p->G; a.R = p->R; a.Nt = p->Nt;
  a.z_lo = (T)p->z_lo; a.dz = (T)p->dz; a.inv_dz = (T)(1.0 / p->dz);
  a.h = (T)(p->dx / p->Nt);
  a.k_over_2pi = (T)(p->k / (2.0 * M_PI));
  a.out_d = (T*)p->rd; a.out_ph = (T*)p->rph; a.out_a = (T*)p->ra;
  a.plane_steps = 0;
  a.pl_d = a.pl_ph = a.pl_a = nullptr;
  a.status = p->status;
  return a;
}

template <typename T>
BracketArgs<T> bracket_args(const swkb_plan* p, const T* d, int* jlo = nullptr,
                            int* jlo_neg = nullptr) {
  return BracketArgs<T>{d, p->Mr, p->NRT, p->G, p->R, p->N, p->TM, p->n_tiles,
                        jlo ? jlo : p->jlo, p->sym, jlo ? jlo_neg : p->jlo_neg, p->status};
}

template <typename T>
ResumArgs<T> resum_args(const swkb_plan* p, const T* d, const T* ph, const T* a,
                        const typename C2<T>::type* c, const int* jlo = nullptr,
                        const int* jlo_neg = nullptr) {
  using V = typename C2<T>::type;
  ResumArgs<T> ra;
  ra.d = d; ra.ph = ph; ra.a = a; ra.jlo = jlo ? jlo : p->jlo;
  ra.jlo_neg = jlo ? jlo_neg : p->jlo_neg;
  ra.c = c;
  ra.cpol = (c == (const typename C2<T>::type*)p->c) ? (const V*)p->cpol : (const V*)p->cpol_plane;
  ra.M = p->M; ra.Mr = p->Mr; ra.sym = p->sym; ra.n_tiles_run = p->n_tiles_run; ra.NRT = p->NRT;
  ra.G = p->G; ra.R = p->R; ra.N = p->N; ra.TM = p->TM;
  ra.PW = p->PW; ra.n_tiles = p->n_tiles; ra.n_groups = p->n_groups;
  ra.modes_per_group = p->modes_per_group; ra.n_max = p->n_max; ra.wcap = p->wcap;
  ra.part = (V*)p->part; ra.status = p->status;
  return ra;
}

template <typename T>
FftArgs<T> fft_args(const swkb_plan* p, bool fuse) {
  using V = typename C2<T>::type;
  FftArgs<T> f;
  f.u = (const V*)p->u; f.tw = (const V*)p->tw; f.Y = (V*)p->Y;
  f.N = p->N; f.N1 = p->N1; f.N2 = p->N2; f.log2N2 = p->log2N2; f.n_max = p->n_max;
  f.mirror = p->mirror;
  f.part = fuse ? (const V*)p->part : nullptr;
  f.n_part = p->n_groups;
  f.sym = p->sym;
  f.W = (const T*)p->W;
  f.inv_N = (T)(1.0 / p->N);
  f.ephi = (const V*)p->ephi_d; f.c = (V*)p->c; f.cpol = (V*)p->cpol;
  return f;
}

template <typename T>
FcModesArgs<T> fc_modes_args(const swkb_plan* p) {
  using V = typename C2<T>::type;
  FcModesArgs<T> f;
  f.u = (const V*)p->u;
  f.n_pat = p->fc_pat; f.stride = p->fc_stride; f.P = p->fc_P; f.Np = p->fc_Np;
  f.n_max = p->n_max; f.M = p->M;
  f.cont = (const double*)p->fc_cont;
  f.tw = (const double2*)p->fc_tw;
  f.ephi = (const V*)p->ephi_d;
  f.inv_Np = 1.0 / p->fc_Np;
  f.np_magic = (unsigned)((1ULL << 32) / (unsigned long long)p->fc_Np);
  f.cf = (V*)p->fc_cf;
  return f;
}

template <typename T>
FcResumArgs<T> fc_resum_args(const swkb_plan* p, const T* d, const T* ph, const T* a,
                             const int* jlo, const void* cf = nullptr) {
  using V = typename C2<T>::type;
  FcResumArgs<T> r;
  r.d = d; r.ph = ph; r.a = a; r.jlo = jlo;
  r.cf = (const V*)(cf ? cf : p->fc_cf);
  r.win_p = p->fc_win_p;
  r.win_s = (const V*)p->fc_win_s;
  r.M = p->M; r.NRT = p->NRT; r.G = p->G; r.R = p->R; r.N = p->N; r.TM = p->TM;
  r.n_tiles = p->n_tiles; r.n_groups = p->n_groups; r.modes_per_group = p->modes_per_group;
  r.n_max = p->n_max; r.wcap = p->wcap; r.Np = p->fc_Np; r.P = p->fc_P;
  r.np_magic = (unsigned)((1ULL << 32) / (unsigned long long)p->fc_Np);
  r.part = (V*)p->part; r.status = p->status;
  return r;
}

// One patch-wise screen (Sec. 2.2): partials -> field, the patches' FC
// modes, rays, brackets, and the sum with per-ray complex amplitudes.
template <typename T>
swkb_status fc_screen(swkb_plan* p, int q, bool u_fresh) {
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream;
  if (!u_fresh) {
    ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, nullptr, 0, 0, (V*)p->u};
    TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
  }
  const FcModesArgs<T> f = fc_modes_args<T>(p);
  TRY(timed(p, SWKB_KERNEL_FFT, 1, [&] { return launch_fc_modes<T>(f, s); }));
  const MarchArgs<T> ma = march_args<T>(p, q);
  const bool multi = p->n_cols > 1;
  const bool march = !(p->reuse_rays && p->rays_ready);
  if (march)
    TRY(timed(p, SWKB_KERNEL_MARCH, 1, [&] { return launch_march<T>(ma, multi, s); }));
  const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->rd);
  if (march) TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
  p->rays_ready = true;
  const FcResumArgs<T> ra = fc_resum_args<T>(p, (const T*)p->rd, (const T*)p->rph,
                                             (const T*)p->ra, p->jlo);
  TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_fc_resum<T>(ra, s); }));
  p->stats.screens += 1;
  return SWKB_OK;
}

template <typename T>
swkb_status launch_screen(swkb_plan* p, int q, bool u_fresh) {
  Range range("swkb_screen");
  if (p->fc) return fc_screen<T>(p, q, u_fresh);
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream;
  // with a two-pass DFT, pass 1 forms the field from the partials itself
  const bool fuse = p->fuse_reduce && !u_fresh && p->N1 > 1 && (p->sym || !p->mirror);
  if (!u_fresh && !fuse) {
    ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, (const T*)p->W, p->mirror, p->sym,
                    (V*)p->u};
    TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
  }
  FftArgs<T> f;
  f.u = (const V*)p->u; f.tw = (const V*)p->tw; f.Y = (V*)p->Y;
  f.N = p->N; f.N1 = p->N1; f.N2 = p->N2; f.log2N2 = p->log2N2; f.n_max = p->n_max;
  f.mirror = p->mirror;
  f.part = fuse ? (const V*)p->part : nullptr;
  f.n_part = p->n_groups;
  f.sym = p->sym;
  f.W = (const T*)p->W;
  f.inv_N = (T)(1.0 / p->N);
  f.ephi = (const V*)p->ephi_d; f.c = (V*)p->c; f.cpol = (V*)p->cpol;
  TRY(timed(p, SWKB_KERNEL_FFT, p->N1 > 1 ? 2 : 1, [&] { return launch_fft<T>(f, s); }));
  const MarchArgs<T> ma = march_args<T>(p, q);
  const bool multi = p->n_cols > 1;
  // a range-independent medium gives every screen the same rays: with
  // reuse_rays they are marched (and bracketed) once per enqueue sequence
  const bool march = !(p->reuse_rays && p->rays_ready);
  if (march)
    TRY(timed(p, SWKB_KERNEL_MARCH, 1, [&] { return launch_march<T>(ma, multi, s); }));
  const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->rd);
  if (march) TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
  p->rays_ready = true;
  const ResumArgs<T> ra = resum_args<T>(p, (const T*)p->rd, (const T*)p->rph, (const T*)p->ra,
                                        (const V*)p->c);
  TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_resum<T>(ra, s); }));
  p->stats.screens += 1;
  return SWKB_OK;
}

template <typename T>
swkb_status reduce_to_u(swkb_plan* p, bool project) {
  using V = typename C2<T>::type;
  // grounded plans sum only the physical half, so their reduction always
  // fills the other half by reflection
  ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, (const T*)p->W,
                  (project || p->sym) ? p->mirror : 0, p->sym, (V*)p->u};
  TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, p->stream); }));
  return SWKB_OK;
}

swkb_status read_status(swkb_plan* p) {
  unsigned bits = 0;
  CK(cudaMemcpyAsync(&bits, p->status, sizeof(unsigned), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  TRY(harvest(p));
  if (bits) {
    CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), p->stream));
    CK(cudaStreamSynchronize(p->stream));
  }
  return status_from_bits(bits);
}

// Enqueue screens q0 .. q0 + n - 1 from the n_z-point field u0 (device,
// complex128).  Each output field (the last one, or every snap-th) goes
// either to out_dev + k n_z (device) or through the staging buffer to
// out_host + k n_z (host).
template <typename T>
swkb_status enqueue(swkb_plan* p, const double* u0, int q0, int n, double* out_dev,
                    double* out_host, int snap) {
  using V = typename C2<T>::type;
  p->rays_ready = false;
  const int off = p->mirror ? p->n_z : 0;
  const size_t nb = 2 * sizeof(double) * p->n_z;
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(u0, p->n_z, p->fc ? p->n_z : p->N, p->mirror, (V*)p->u,
                                        p->stream); }));
  bool fresh = true;
  int k = 0;
  auto emit = [&](int idx) -> swkb_status {
    double* dst = out_dev ? out_dev + 2 * (size_t)idx * p->n_z : p->io;
    TRY(timed(p, SWKB_KERNEL_OUTPUT, 1,
              [&] { return launch_output<T>((const V*)p->u, off, p->n_z, dst, p->stream); }));
    if (!out_dev)
      CK(cudaMemcpyAsync(out_host + 2 * (size_t)idx * p->n_z, p->io, nb, cudaMemcpyDeviceToHost,
                         p->stream));
    return SWKB_OK;
  };
  for (int q = q0; q < q0 + n; ++q) {
    TRY(launch_screen<T>(p, q, fresh));
    fresh = false;
    if (snap > 0 && (q - q0 + 1) % snap == 0) {
      TRY(reduce_to_u<T>(p, true));
      fresh = true;
      TRY(emit(k++));
    }
  }
  if (snap <= 0) {
    if (!fresh) TRY(reduce_to_u<T>(p, true));
    TRY(emit(0));
  }
  return SWKB_OK;
}

// One screen of the overlapped sequence: rays of screen q into ray-buffer set
// b on ray_stream, modes of the field on the plan stream, then brackets and
// sum once the rays are there.  ev_free[b] must have been recorded (set free).
template <typename T>
swkb_status overlapped_screen(swkb_plan* p, int q, int b, bool fresh) {
  Range range("swkb_screen");
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream, sr = p->ray_stream;
  T* rd[2] = {(T*)p->rd, (T*)p->rd1};
  T* rph[2] = {(T*)p->rph, (T*)p->rph1};
  T* ra[2] = {(T*)p->ra, (T*)p->ra1};
  int* jlo[2] = {p->jlo, p->jlo1};
  int* jneg[2] = {p->jlo_neg, p->jlo_neg1};
  const bool multi = p->n_cols > 1;
  // rays of screen q
  CK(cudaStreamWaitEvent(sr, p->ev_free[b], 0));
  MarchArgs<T> ma = march_args<T>(p, q);
  ma.out_d = rd[b]; ma.out_ph = rph[b]; ma.out_a = ra[b];
  TRY(timed_on(p, sr, SWKB_KERNEL_MARCH, 1, [&] { return launch_march<T>(ma, multi, sr); }));
  CK(cudaEventRecord(p->ev_rays[b], sr));
  if (p->fc) {
    if (!fresh) {
      ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, nullptr, 0, 0, (V*)p->u};
      TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
    }
    const FcModesArgs<T> fm = fc_modes_args<T>(p);
    TRY(timed(p, SWKB_KERNEL_FFT, 1, [&] { return launch_fc_modes<T>(fm, s); }));
    CK(cudaStreamWaitEvent(s, p->ev_rays[b], 0));
    const BracketArgs<T> br = bracket_args<T>(p, rd[b], jlo[b], jneg[b]);
    TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(br, s); }));
    const FcResumArgs<T> rs = fc_resum_args<T>(p, rd[b], rph[b], ra[b], jlo[b]);
    TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_fc_resum<T>(rs, s); }));
    CK(cudaEventRecord(p->ev_free[b], s));
    p->stats.screens += 1;
    return SWKB_OK;
  }
  // modes of screen q (pass 1 forms the field from the partials itself)
  const bool fuse = p->fuse_reduce && !fresh && p->N1 > 1 && (p->sym || !p->mirror);
  if (!fresh && !fuse) {
    ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, (const T*)p->W, p->mirror, p->sym,
                    (V*)p->u};
    TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
  }
  FftArgs<T> f;
  f.u = (const V*)p->u; f.tw = (const V*)p->tw; f.Y = (V*)p->Y;
  f.N = p->N; f.N1 = p->N1; f.N2 = p->N2; f.log2N2 = p->log2N2; f.n_max = p->n_max;
  f.mirror = p->mirror;
  f.part = fuse ? (const V*)p->part : nullptr;
  f.n_part = p->n_groups;
  f.sym = p->sym;
  f.W = (const T*)p->W;
  f.inv_N = (T)(1.0 / p->N);
  f.ephi = (const V*)p->ephi_d; f.c = (V*)p->c; f.cpol = (V*)p->cpol;
  TRY(timed(p, SWKB_KERNEL_FFT, p->N1 > 1 ? 2 : 1, [&] { return launch_fft<T>(f, s); }));
  // brackets and sum of screen q, once its rays are there (the ray stream
  // goes on with the next march)
  CK(cudaStreamWaitEvent(s, p->ev_rays[b], 0));
  const BracketArgs<T> br = bracket_args<T>(p, rd[b], jlo[b], jneg[b]);
  TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(br, s); }));
  const ResumArgs<T> rs = resum_args<T>(p, rd[b], rph[b], ra[b], (const V*)p->c, jlo[b],
                                        jneg[b]);
  TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_resum<T>(rs, s); }));
  CK(cudaEventRecord(p->ev_free[b], s));
  p->stats.screens += 1;
  return SWKB_OK;
}

// enqueue() with the rays on a second stream.  A screen's rays depend only on
// the medium and the mode angles, never on the field, so the march of screen
// q (into ray-buffer set (q - q0) % 2, on ray_stream) runs beside the DFT of
// screen q and the bracket and resummation of screen q - 1 on the plan stream.
// The bracket of screen q waits for its set's "rays" event; the march of
// screen q + 2 waits for the "free" event recorded after the resummation of
// screen q, the last reader of that set.  Same kernels and
// arguments as enqueue(): the fields are bit-identical.
template <typename T>
swkb_status enqueue_overlapped(swkb_plan* p, const double* u0, int q0, int n, double* out_dev,
                               double* out_host, int snap) {
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream;
  const int off = p->mirror ? p->n_z : 0;
  const size_t nb = 2 * sizeof(double) * p->n_z;
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(u0, p->n_z, p->fc ? p->n_z : p->N, p->mirror, (V*)p->u,
                                        s); }));
  // both sets start free (this also forks ray_stream from the plan stream)
  CK(cudaEventRecord(p->ev_free[0], s));
  CK(cudaEventRecord(p->ev_free[1], s));
  bool fresh = true;
  int k = 0;
  auto emit = [&](int idx) -> swkb_status {
    double* dst = out_dev ? out_dev + 2 * (size_t)idx * p->n_z : p->io;
    TRY(timed(p, SWKB_KERNEL_OUTPUT, 1,
              [&] { return launch_output<T>((const V*)p->u, off, p->n_z, dst, s); }));
    if (!out_dev)
      CK(cudaMemcpyAsync(out_host + 2 * (size_t)idx * p->n_z, p->io, nb, cudaMemcpyDeviceToHost,
                         s));
    return SWKB_OK;
  };
  for (int q = q0; q < q0 + n; ++q) {
    TRY(overlapped_screen<T>(p, q, (q - q0) & 1, fresh));
    fresh = false;
    if (snap > 0 && (q - q0 + 1) % snap == 0) {
      TRY(reduce_to_u<T>(p, true));
      fresh = true;
      TRY(emit(k++));
    }
  }
  if (snap <= 0) {
    if (!fresh) TRY(reduce_to_u<T>(p, true));
    TRY(emit(0));
  }
  return SWKB_OK;
}

// Fields on the planes x_q + j dx / P (j = 1..P) of screens q0 .. q0 + n - 1,
// rows ordered (screen, plane); the last plane of a screen is the screen's
// field, the planes before it are the ray field between screens: the
// screen's modes, its rays stopped after j N_t / P RK4 steps, the same
// interpolation and sum with the range-phase carry of that plane, and no
// absorber.  Uses the inner-plane buffers (P <= the plan's planes option).
// enqueue_planes() for a patch-wise plan: the patches' modes once per
// screen, carried to each inner plane by exp(i k (j/P - 1) dx Pbar_n).
template <typename T>
swkb_status enqueue_planes_fc(swkb_plan* p, const double* u0, int q0, int n, int P,
                              double* out_dev, double* out_host) {
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream;
  p->rays_ready = false;
  const size_t nb = 2 * sizeof(double) * p->n_z;
  const size_t rays = (size_t)p->NRT * p->Mr;
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(u0, p->n_z, p->n_z, 0, (V*)p->u, s); }));
  int row = 0;
  auto emit = [&]() -> swkb_status {
    const int idx = row++;
    double* dst = out_dev ? out_dev + 2 * (size_t)idx * p->n_z : p->io;
    TRY(timed(p, SWKB_KERNEL_OUTPUT, 1,
              [&] { return launch_output<T>((const V*)p->u, 0, p->n_z, dst, s); }));
    if (!out_dev)
      CK(cudaMemcpyAsync(out_host + 2 * (size_t)idx * p->n_z, p->io, nb, cudaMemcpyDeviceToHost,
                         s));
    return SWKB_OK;
  };
  auto reduce = [&]() -> swkb_status {
    ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, nullptr, 0, 0, (V*)p->u};
    TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
    return SWKB_OK;
  };
  for (int q = q0; q < q0 + n; ++q) {
    const FcModesArgs<T> f = fc_modes_args<T>(p);
    TRY(timed(p, SWKB_KERNEL_FFT, 1, [&] { return launch_fc_modes<T>(f, s); }));
    MarchArgs<T> ma = march_args<T>(p, q);
    if (P > 1) {
      ma.plane_steps = p->Nt / P;
      ma.pl_d = (T*)p->pl_d; ma.pl_ph = (T*)p->pl_ph; ma.pl_a = (T*)p->pl_a;
    }
    const bool multi = p->n_cols > 1;
    TRY(timed(p, SWKB_KERNEL_MARCH, 1, [&] { return launch_march<T>(ma, multi, s); }));
    for (int j = 1; j < P; ++j) {
      const size_t o = (size_t)(j - 1) * rays;
      const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->pl_d + o);
      TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
      const V* fj = (const V*)p->ephi_pl + (size_t)(j - 1) * p->M;
      TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] {
        return launch_fc_cscale<T>((const V*)p->fc_cf, fj, (V*)p->fc_cf_plane, p->fc_P, p->M, s);
      }));
      const FcResumArgs<T> ra = fc_resum_args<T>(p, (const T*)p->pl_d + o,
                                                 (const T*)p->pl_ph + o, (const T*)p->pl_a + o,
                                                 p->jlo, p->fc_cf_plane);
      TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_fc_resum<T>(ra, s); }));
      TRY(reduce());
      TRY(emit());
    }
    const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->rd);
    TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
    const FcResumArgs<T> ra = fc_resum_args<T>(p, (const T*)p->rd, (const T*)p->rph,
                                               (const T*)p->ra, p->jlo);
    TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_fc_resum<T>(ra, s); }));
    TRY(reduce());
    TRY(emit());
    p->stats.screens += 1;
  }
  return SWKB_OK;
}

template <typename T>
swkb_status enqueue_planes(swkb_plan* p, const double* u0, int q0, int n, int P,
                           double* out_dev, double* out_host) {
  if (p->fc) return enqueue_planes_fc<T>(p, u0, q0, n, P, out_dev, out_host);
  using V = typename C2<T>::type;
  cudaStream_t s = p->stream;
  p->rays_ready = false;
  const int off = p->mirror ? p->n_z : 0;
  const size_t nb = 2 * sizeof(double) * p->n_z;
  const size_t rays = (size_t)p->NRT * p->Mr;
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(u0, p->n_z, p->N, p->mirror, (V*)p->u, s); }));
  int row = 0;
  auto emit = [&]() -> swkb_status {
    const int idx = row++;
    double* dst = out_dev ? out_dev + 2 * (size_t)idx * p->n_z : p->io;
    TRY(timed(p, SWKB_KERNEL_OUTPUT, 1,
              [&] { return launch_output<T>((const V*)p->u, off, p->n_z, dst, s); }));
    if (!out_dev)
      CK(cudaMemcpyAsync(out_host + 2 * (size_t)idx * p->n_z, p->io, nb, cudaMemcpyDeviceToHost,
                         s));
    return SWKB_OK;
  };
  // partials -> field on the whole period (grounded: reflection fill), with
  // or without the absorber
  auto reduce = [&](const T* W) -> swkb_status {
    ReduceArgs<T> r{(const V*)p->part, p->n_groups, p->N, W, p->mirror, p->sym, (V*)p->u};
    TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] { return launch_reduce<T>(r, s); }));
    return SWKB_OK;
  };
  for (int q = q0; q < q0 + n; ++q) {
    FftArgs<T> f;
    f.u = (const V*)p->u; f.tw = (const V*)p->tw; f.Y = (V*)p->Y;
    f.N = p->N; f.N1 = p->N1; f.N2 = p->N2; f.log2N2 = p->log2N2; f.n_max = p->n_max;
    f.mirror = p->mirror;
    f.part = nullptr;
    f.n_part = p->n_groups;
    f.sym = p->sym;
    f.W = (const T*)p->W;
    f.inv_N = (T)(1.0 / p->N);
    f.ephi = (const V*)p->ephi_d; f.c = (V*)p->c; f.cpol = (V*)p->cpol;
    TRY(timed(p, SWKB_KERNEL_FFT, p->N1 > 1 ? 2 : 1, [&] { return launch_fft<T>(f, s); }));
    MarchArgs<T> ma = march_args<T>(p, q);
    if (P > 1) {
      ma.plane_steps = p->Nt / P;
      ma.pl_d = (T*)p->pl_d; ma.pl_ph = (T*)p->pl_ph; ma.pl_a = (T*)p->pl_a;
    }
    const bool multi = p->n_cols > 1;
    TRY(timed(p, SWKB_KERNEL_MARCH, 1, [&] { return launch_march<T>(ma, multi, s); }));
    for (int j = 1; j < P; ++j) {
      const size_t o = (size_t)(j - 1) * rays;
      const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->pl_d + o);
      TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
      // c_n of plane j: the screen's c_n (carried over dx) times exp(i k (j/P - 1) dx P_bar_n)
      const V* fj = (const V*)p->ephi_pl + (size_t)(j - 1) * p->M;
      TRY(timed(p, SWKB_KERNEL_REDUCE, 1, [&] {
        return launch_cscale<T>((const V*)p->c, fj, (V*)p->c_plane, (V*)p->cpol_plane, p->M, s);
      }));
      const ResumArgs<T> ra = resum_args<T>(p, (const T*)p->pl_d + o, (const T*)p->pl_ph + o,
                                            (const T*)p->pl_a + o, (const V*)p->c_plane);
      TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_resum<T>(ra, s); }));
      TRY(reduce(nullptr));
      TRY(emit());
    }
    const BracketArgs<T> b = bracket_args<T>(p, (const T*)p->rd);
    TRY(timed(p, SWKB_KERNEL_BRACKET, 1, [&] { return launch_bracket<T>(b, s); }));
    const ResumArgs<T> ra = resum_args<T>(p, (const T*)p->rd, (const T*)p->rph, (const T*)p->ra,
                                          (const V*)p->c);
    TRY(timed(p, SWKB_KERNEL_RESUM, 1, [&] { return launch_resum<T>(ra, s); }));
    TRY(reduce((const T*)p->W));
    TRY(emit());
    p->stats.screens += 1;
  }
  return SWKB_OK;
}

// Range-phase factors exp(i k (j/P - 1) dx P_bar_n) of the inner planes
// j = 1..P-1, formed in FP64 and reduced mod 2 pi on the host.
template <typename T>
swkb_status upload_plane_phases(swkb_plan* p, int P) {
  std::vector<T> f(2 * (size_t)(P - 1) * p->M);
  for (int j = 1; j < P; ++j)
    for (int i = 0; i < p->M; ++i) {
      const double phi = fmod(p->k * p->dx * ((double)j / P - 1.0) * p->pbar[i], 2.0 * M_PI);
      f[2 * ((size_t)(j - 1) * p->M + i)] = (T)cos(phi);
      f[2 * ((size_t)(j - 1) * p->M + i) + 1] = (T)sin(phi);
    }
  CK(cudaMemcpyAsync(p->ephi_pl, f.data(), f.size() * sizeof(T), cudaMemcpyHostToDevice,
                     p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return SWKB_OK;
}

void drop_graphs(swkb_plan* p) {
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
}

// Propagate as one CUDA graph: captured on first use for this (screen range,
// buffers, timing) and replayed afterwards, so a whole propagation costs one
// launch on the host.  Host-side copies stay outside the graph.
template <typename T>
swkb_status run_graph(swkb_plan* p, const double* u0, int q0, int n, double* dst, int snap) {
  swkb_plan::Graph* g = nullptr;
  for (auto& e : p->graphs)
    if (e.q0 == q0 && e.n == n && e.snap == snap && e.in == u0 && e.out == dst &&
        e.timing == timing_key(p) && e.every == p->timing_every)
      g = &e;
  if (!g) {
    if (p->graphs.size() >= 8) drop_graphs(p);
    const swkb_plan_stats before = p->stats;
    p->marks.clear();
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    swkb_status st = overlapped(p) ? enqueue_overlapped<T>(p, u0, q0, n, dst, nullptr, snap)
                                   : enqueue<T>(p, u0, q0, n, dst, nullptr, snap);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->stream, &graph);
    if (st == SWKB_OK && ec != cudaSuccess)
      st = fail(SWKB_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ec));
    cudaGraphExec_t exec = nullptr;
    if (st == SWKB_OK) {
      const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      if (ei != cudaSuccess)
        st = fail(SWKB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ei));
    }
    if (graph) cudaGraphDestroy(graph);
    swkb_plan::Graph e{q0, n, snap, timing_key(p), p->timing_every, u0, dst, exec, p->marks, {}};
    e.delta.launches = p->stats.launches - before.launches;
    e.delta.screens = p->stats.screens - before.screens;
    for (int kk = 0; kk < SWKB_KERNEL_KINDS; ++kk) {
      e.delta.kernel_launches[kk] = p->stats.kernel_launches[kk] - before.kernel_launches[kk];
      e.delta.kernel_timed[kk] = p->stats.kernel_timed[kk] - before.kernel_timed[kk];
    }
    p->stats = before;
    p->marks.clear();
    if (st != SWKB_OK) {
      cudaGetLastError();
      return st;
    }
    p->graphs.push_back(e);
    g = &p->graphs.back();
  }
  CK(cudaGraphLaunch(g->exec, p->stream));
  p->marks.insert(p->marks.end(), g->marks.begin(), g->marks.end());
  p->stats.launches += g->delta.launches;
  p->stats.screens += g->delta.screens;
  for (int kk = 0; kk < SWKB_KERNEL_KINDS; ++kk) {
    p->stats.kernel_launches[kk] += g->delta.kernel_launches[kk];
    p->stats.kernel_timed[kk] += g->delta.kernel_timed[kk];
  }
  return SWKB_OK;
}

template <typename T>
swkb_status run(swkb_plan* p, const double* u0, int q0, int n, double* out_dev, double* out_host,
                int snap) {
  // graphs need a capturable stream and device-side outputs (snapshots to
  // host memory interleave copies, which run directly instead)
  if (p->use_graphs && p->stream != nullptr && (out_dev || snap <= 0)) {
    double* dst = out_dev ? out_dev : p->io;
    TRY(run_graph<T>(p, u0, q0, n, dst, snap));
    if (!out_dev)
      CK(cudaMemcpyAsync(out_host, p->io, 2 * sizeof(double) * p->n_z, cudaMemcpyDeviceToHost,
                         p->stream));
    return read_status(p);
  }
  TRY(overlapped(p) ? enqueue_overlapped<T>(p, u0, q0, n, out_dev, out_host, snap)
                    : enqueue<T>(p, u0, q0, n, out_dev, out_host, snap));
  return read_status(p);
}

template <typename T>
swkb_status debug_screen(swkb_plan* p, int q, const double* u_full, double* c, double* delta,
                         double* r, double* a, double* u_next) {
  using V = typename C2<T>::type;
  const int N = p->N, M = p->M, NRT = p->NRT;
  CK(cudaMemcpyAsync(p->io, u_full, 2 * sizeof(double) * N, cudaMemcpyHostToDevice, p->stream));
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(p->io, N, N, 0, (V*)p->u, p->stream); }));
  p->rays_ready = false;
  TRY(launch_screen<T>(p, q, true));
  TRY(reduce_to_u<T>(p, false));
  std::vector<V> hc(M), hu(N);
  const int Mr = p->Mr;
  std::vector<T> hd((size_t)NRT * Mr), hph((size_t)NRT * Mr), ha((size_t)NRT * Mr);
  CK(cudaMemcpyAsync(hc.data(), p->c, sizeof(V) * M, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(hu.data(), p->u, sizeof(V) * N, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(hd.data(), p->rd, sizeof(T) * hd.size(), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(hph.data(), p->rph, sizeof(T) * hd.size(), cudaMemcpyDeviceToHost, p->stream));
  CK(cudaMemcpyAsync(ha.data(), p->ra, sizeof(T) * hd.size(), cudaMemcpyDeviceToHost, p->stream));
  TRY(read_status(p));
  if (c) {
    for (int i = 0; i < M; ++i) {   // divide out exp(i Phi_n)
      const double er = p->ephi[2 * i], ei = p->ephi[2 * i + 1];
      const double xr = hc[i].x, xi = hc[i].y;
      c[2 * i] = xr * er + xi * ei;
      c[2 * i + 1] = xi * er - xr * ei;
    }
  }
  const double two_pi_over_k = 2.0 * M_PI / p->k;
  for (int i = 0; i < M; ++i) {
    const int n = i - p->n_max;
    const bool mir = p->sym && n < 0;
    const int col = p->sym ? (n < 0 ? -n : n) : i;
    for (int j = 0; j < NRT; ++j) {
      const size_t dst = (size_t)i * NRT + j;
      // grounded plans march n >= 0; ray j of mode -n mirrors ray NRT - j of
      // mode n (ray 0 of a mirrored family has no partner: NaN)
      const int js = mir ? NRT - j : j;
      if (js >= NRT) {
        if (delta) delta[dst] = NAN;
        if (r) r[dst] = NAN;
        if (a) a[dst] = NAN;
        continue;
      }
      const size_t src = (size_t)js * Mr + col;
      const double g = (double)((long long)(js - p->G) * p->R) + (double)hd[src];
      if (delta) delta[dst] = mir ? p->N - g : g;
      if (r) r[dst] = (double)hph[src] * two_pi_over_k + p->dx * p->pbar[i];
      if (a) a[dst] = (double)ha[src];
    }
  }
  if (u_next) {
    for (int m = 0; m < N; ++m) {
      u_next[2 * m] = hu[m].x;
      u_next[2 * m + 1] = hu[m].y;
    }
  }
  return SWKB_OK;
}

void release(swkb_plan* p) {
  if (!p) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(p->device);
  // a sequence that failed between a march and the wait that joins it may
  // leave work on the ray stream: finish it before its buffers go
  if (p->ray_stream) cudaStreamSynchronize(p->ray_stream);
  drop_graphs(p);
  for (void* ptr : p->allocs) cudaFree(ptr);
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    if (p->ev_rays[b]) cudaEventDestroy(p->ev_rays[b]);
    if (p->ev_free[b]) cudaEventDestroy(p->ev_free[b]);
  }
  if (p->ray_stream) cudaStreamDestroy(p->ray_stream);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  cudaSetDevice(cur);
  delete p;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void swkb_options_default(swkb_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = SWKB_FP64;
  o->theta_max = M_PI / 6.0;
  o->n_max = 0;
  o->ray_stride = 1;
  o->rk4_steps = 8;
  o->absorber_frac = 0.0;
  o->autotune = 0;
  o->cuda_stream = nullptr;
  o->device = 0;
  o->reuse_rays = 0;
  o->planes = 0;
}

const char* swkb_last_error(void) { return g_err.c_str(); }

const char* swkb_status_string(swkb_status s) {
  switch (s) {
    case SWKB_OK: return "ok";
    case SWKB_ERR_INVALID_ARG: return "invalid argument";
    case SWKB_ERR_OOM: return "out of device memory";
    case SWKB_ERR_CAUSTIC: return "caustic between screens";
    case SWKB_ERR_TURNING: return "turning point on a ray";
    case SWKB_ERR_RANGE: return "ray outside the table or the screen";
    case SWKB_ERR_CUDA: return "CUDA error";
    case SWKB_ERR_TIMEOUT: return "timeout";
    case SWKB_ERR_AGAIN: return "queue full";
    case SWKB_NOT_READY: return "not ready";
    case SWKB_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

// Launch shapes chosen per plan: resummation tile (PW points per lane, tile
// of 32 PW grid points), resummation CTAs per SM (mode groups), DFT split
// N = N1 N2.
struct Tiling {
  int PW, ctas_per_sm, N1;
};

bool valid_tiling(const swkb_plan* p, const Tiling& t) {
  if (t.PW != 2 && t.PW != 4 && t.PW != 8 && t.PW != 16) return false;
  if (p->fc && (t.PW > 8 || p->N % (32 * t.PW))) return false;
  if (32 * t.PW > (p->sym ? p->N / 2 : p->N)) return false;
  if (t.N1 < 1 || t.N1 > 64 || (t.N1 & (t.N1 - 1)) || t.N1 > p->N / 32) return false;
  return t.ctas_per_sm >= 1;
}

Tiling default_tiling(const swkb_plan* p) {
  Tiling t;
  t.PW = p->R >= 8 ? 8 : (p->R >= 2 ? 4 : 2);
  while (32 * t.PW > (p->sym ? p->N / 2 : p->N) || (p->fc && p->N % (32 * t.PW))) t.PW /= 2;
  // patch-wise plans are not autotuned: many short mode groups keep the
  // last wave of their sum short (measured on the open lens, N_z = 131072:
  // 0.31 ms per sum with 2 groups, 0.26 with 8)
  t.ctas_per_sm = p->fc ? 24 : 6;
  // N1 ~ sqrt(M): pass 1 costs N N1, pass 2 M N2
  t.N1 = 1;
  while (t.N1 * t.N1 * 2 < p->M && t.N1 < p->N / 32 && t.N1 < 64) t.N1 *= 2;
  return t;
}

std::vector<Tiling> tiling_candidates(const swkb_plan* p) {
  const Tiling d = default_tiling(p);
  std::vector<Tiling> out;
  for (int pw : {d.PW / 2, d.PW, d.PW * 2})
    for (int c : {4, 6, 8, 12})
      for (int n1 : {d.N1, d.N1 * 2}) {
        const Tiling t{pw, c, n1};
        if (valid_tiling(p, t)) out.push_back(t);
      }
  return out;
}

void apply_tiling(swkb_plan* p, const Tiling& t) {
  p->PW = t.PW;
  p->TM = 32 * t.PW;
  p->n_tiles = p->N / p->TM;
  p->n_tiles_run = p->sym ? p->n_tiles / 2 + 1 : p->n_tiles;
  // rays per tile window: up to 4x compression (patch-wise plans: exactly,
  // which keeps six FP32 sums of 4 warps within an SM's shared memory)
  p->wcap = 4 * p->TM / p->R + (p->fc ? 4 : 8);
  p->ctas_per_sm = t.ctas_per_sm;
  const int target_ctas = p->sms * t.ctas_per_sm;
  p->n_groups = std::max(1, std::min(p->M, (target_ctas + p->n_tiles_run - 1) / p->n_tiles_run));
  p->modes_per_group = (p->M + p->n_groups - 1) / p->n_groups;
  p->n_groups = (p->M + p->modes_per_group - 1) / p->modes_per_group;
  p->N1 = t.N1;
  p->N2 = p->N / p->N1;
  p->log2N2 = ilog2(p->N2);
}

// Validate the arguments and derive every size of the plan (host only).
swkb_status configure(swkb_plan* p, const swkb_profile* prof, double k, const swkb_domain* dom,
                      int32_t n_z, double screen_dx, const swkb_options& opt) {
  if (!prof || !dom) return fail(SWKB_ERR_INVALID_ARG, "profile or domain is NULL");
  if (!(k > 0) || !std::isfinite(k)) return fail(SWKB_ERR_INVALID_ARG, "k must be > 0");
  if (!(dom->z_b > dom->z_a)) return fail(SWKB_ERR_INVALID_ARG, "need z_b > z_a");
  if (!(screen_dx > 0)) return fail(SWKB_ERR_INVALID_ARG, "screen spacing must be > 0");
  if (dom->bc < SWKB_BC_PERIODIC || dom->bc > SWKB_BC_OPEN)
    return fail(SWKB_ERR_INVALID_ARG, "unknown boundary condition %d", dom->bc);
  if (opt.precision != SWKB_FP64 && opt.precision != SWKB_MIXED)
    return fail(SWKB_ERR_INVALID_ARG, "unknown precision %d", opt.precision);
  if (prof->n_cols < 1 || prof->n_p < 3 || !(prof->dz_p > 0) || !prof->x_cols || !prof->eps ||
      !prof->eps_z || !prof->eps_zz)
    return fail(SWKB_ERR_INVALID_ARG, "malformed profile table");
  for (int c = 1; c < prof->n_cols; ++c)
    if (!(prof->x_cols[c] >= prof->x_cols[c - 1]))
      return fail(SWKB_ERR_INVALID_ARG, "x_cols must be non-decreasing");
  const size_t nt = (size_t)prof->n_cols * prof->n_p;
  for (size_t i = 0; i < nt; ++i)
    if (!std::isfinite(prof->eps[i]) || !std::isfinite(prof->eps_z[i]) ||
        !std::isfinite(prof->eps_zz[i]))
      return fail(SWKB_ERR_INVALID_ARG, "profile table has non-finite entries");
  p->precision = opt.precision;
  p->bc = dom->bc;
  p->mirror = dom->bc == SWKB_BC_NEUMANN ? 1 : (dom->bc == SWKB_BC_DIRICHLET ? -1 : 0);
  p->k = k; p->z_a = dom->z_a; p->z_b = dom->z_b; p->x0 = dom->x0; p->dx = screen_dx;
  p->n_z = n_z;
  const double H = dom->z_b - dom->z_a;
  p->fc = dom->bc == SWKB_BC_OPEN;
  if (p->fc) {
    // patch-wise continuation: the rays and the sum cover n_z rounded up to a
    // multiple of 64 (whole resummation tiles of 64, 128 or 256 points that
    // divide it); the extra points belong to no patch
    p->fc_pat = opt.fc_patch;
    p->fc_ov = opt.fc_overlap;
    p->fc_stride = p->fc_pat - p->fc_ov;
    if (n_z < 64 || n_z > (1 << 20) - 256)
      return fail(SWKB_ERR_INVALID_ARG, "n_z %d must be in [64, 2^20 - 256]", n_z);
    if (p->fc_ov < 2 || p->fc_pat < 2 * p->fc_ov || p->fc_pat < 16 || p->fc_pat > n_z ||
        (n_z - p->fc_pat) % p->fc_stride)
      return fail(SWKB_ERR_INVALID_ARG,
                  "patches (fc_patch %d, fc_overlap %d) must satisfy 2 <= fc_overlap, "
                  "2 fc_overlap <= fc_patch, 16 <= fc_patch <= n_z and tile n_z = %d exactly",
                  p->fc_pat, p->fc_ov, n_z);
    p->fc_Np = p->fc_pat + FC_CONT_ROWS;
    if (p->fc_Np > 2048)
      return fail(SWKB_ERR_INVALID_ARG, "fc_patch + %d = %d exceeds 2048", FC_CONT_ROWS,
                  p->fc_Np);
    p->fc_P = (n_z - p->fc_pat) / p->fc_stride + 1;
    if (opt.absorber_frac != 0.0)
      return fail(SWKB_ERR_INVALID_ARG, "patch-wise plans take no absorber");
    p->N = (n_z + 63) / 64 * 64;
    p->L = p->fc_Np * (H / n_z);
  } else {
    p->N = p->mirror ? 2 * n_z : n_z;
    if (n_z < 1 || !is_pow2(p->N) || p->N < 64 || p->N > (1 << 20))
      return fail(SWKB_ERR_INVALID_ARG, "FFT length %d must be a power of two in [64, 2^20]",
                  p->N);
    p->L = p->mirror ? 2 * H : H;
  }
  p->dz = H / n_z;
  p->z_lo = p->mirror ? dom->z_a - H : dom->z_a;
  const double lam = 2.0 * M_PI / k;
  if (opt.n_max > 0) p->n_max = opt.n_max;
  else p->n_max = (int)floor(sin(opt.theta_max) * p->L / lam * (1.0 + 1e-12));
  p->n_max = std::min(p->n_max, (p->fc ? p->fc_Np : p->N) / 2 - 1);
  if (p->n_max < 0) return fail(SWKB_ERR_INVALID_ARG, "negative theta_max or n_max");
  p->M = 2 * p->n_max + 1;
  p->R = opt.ray_stride;
  if (p->R < 1 || p->N % p->R) return fail(SWKB_ERR_INVALID_ARG, "ray stride must divide N");
  p->N_r = p->N / p->R;
  p->Nt = opt.rk4_steps;
  if (p->Nt < 1 || p->Nt > 4096) return fail(SWKB_ERR_INVALID_ARG, "rk4_steps out of range");
  const double kmax = p->n_max * lam / p->L;
  if (!(kmax < 1.0)) return fail(SWKB_ERR_INVALID_ARG, "kept modes reach grazing angle");
  const double tan_t = kmax / sqrt(1.0 - kmax * kmax);
  p->G = (int)ceil(screen_dx * tan_t / (p->R * p->dz) - 1e-9) + 3;
  p->NRT = p->N_r + 2 * p->G;
  p->absorber_frac = opt.absorber_frac;
  if (!(p->absorber_frac >= 0 && p->absorber_frac < 1))
    return fail(SWKB_ERR_INVALID_ARG, "absorber_frac must be in [0, 1)");
  // medium
  p->n_cols = prof->n_cols; p->n_p = prof->n_p; p->n_int = prof->n_p - 1;
  p->z0p = prof->z0_p; p->dzp = prof->dz_p;
  p->x_cols.assign(prof->x_cols, prof->x_cols + prof->n_cols);
  const double ztop = p->z0p + p->dzp * (p->n_p - 1);
  if (p->mirror) {
    if (fabs(p->z0p - p->z_a) > 1e-9 * (1.0 + fabs(p->z_a)))
      return fail(SWKB_ERR_INVALID_ARG, "grounded domains need the table to start at z_a");
    double mx = 0;
    for (size_t i = 0; i < nt; ++i) mx = std::max(mx, fabs(prof->eps_z[i]));
    for (int c = 0; c < p->n_cols; ++c)
      if (fabs(prof->eps_z[(size_t)c * p->n_p]) > 1e-12 * (1.0 + mx))
        return fail(SWKB_ERR_INVALID_ARG, "grounded domains need eps_z = 0 at z_a");
  }
  // the FP32 march finds table intervals with a round-down add (exact below 2^22)
  if (p->precision != SWKB_FP64 && (long long)(p->mirror ? 2 : 1) * p->n_int >= (1LL << 22))
    return fail(SWKB_ERR_INVALID_ARG, "permittivity table has too many intervals for FP32 plans");
  {
    const double reach = 1.5 * screen_dx * tan_t + 2.0 * p->dzp;
    const double s_first = p->z_lo - (double)p->G * p->R * p->dz;
    const double s_last = p->z_lo + (double)(p->NRT - 1 - p->G) * p->R * p->dz;
    double lo = s_first - reach, hi = s_last + reach;
    if (p->mirror) {
      hi = p->z_a + std::max(fabs(lo - p->z_a), fabs(hi - p->z_a));
      lo = p->z_a;
    }
    if (lo < p->z0p - 1e-9 || hi > ztop + 1e-9)
      return fail(SWKB_ERR_INVALID_ARG,
                  "permittivity table covers [%g, %g] but rays may reach [%g, %g]", p->z0p,
                  ztop, lo, hi);
  }
  {
    const double zm = 0.5 * (p->z_a + p->z_b);
    long long im = llround((zm - p->z0p) / p->dzp);
    im = std::min<long long>(std::max<long long>(im, 0), p->n_p - 1);
    p->eps_ref = prof->eps[im];
    if (!(p->eps_ref - kmax * kmax > 0))
      return fail(SWKB_ERR_INVALID_ARG, "steepest kept mode is evanescent at eps_ref");
  }
  p->pieces = p->precision == SWKB_FP64 ? 0 : pieces_for(p, prof);
  if (p->n_cols > 1) {
    const double q_end = ceil((p->x_cols.back() - p->x0) / p->dx);
    p->stage_rows = (int)std::min(std::max(q_end, 0.0), 1e6) + 1;
  }
  // grounded domains: mode -n is the mirror image of mode n and the field
  // is even / odd, so only n >= 0 is marched and only z >= z_a summed
  p->sym = p->mirror != 0;
  p->Mr = p->sym ? p->n_max + 1 : p->M;
  p->device = opt.device;
  CK(cudaSetDevice(p->device));
  CK(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));
  p->autotune = opt.autotune != 0 && !p->fc;
  p->reuse_rays = opt.reuse_rays != 0 && p->n_cols == 1;
  // rays on a second stream unless they are reused (SWKB_OVERLAP=0: one
  // stream, one ray-buffer set)
  {
    const char* oe = getenv("SWKB_OVERLAP");
    p->overlap = !(oe && oe[0] == '0') && !p->reuse_rays;
  }
  p->planes = opt.planes > 1 ? opt.planes : 0;
  if (p->planes && (p->planes > p->Nt || p->Nt % p->planes))
    return fail(SWKB_ERR_INVALID_ARG, "planes (%d) must divide rk4_steps (%d)", p->planes, p->Nt);
  Tiling def = default_tiling(p);
  if (opt.tile_points != 0 || opt.ctas_per_sm != 0 || opt.fft_n1 != 0) {
    const Tiling t{opt.tile_points / 32, opt.ctas_per_sm, opt.fft_n1};
    if (opt.tile_points % 32 || opt.ctas_per_sm > 1024 || !valid_tiling(p, t))
      return fail(SWKB_ERR_INVALID_ARG,
                  "launch shapes (tile_points %d, ctas_per_sm %d, fft_n1 %d) are not valid for "
                  "this plan", opt.tile_points, opt.ctas_per_sm, opt.fft_n1);
    def = t;
    p->autotune = false;
  }
  apply_tiling(p, def);
  {
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    const bool f64 = p->precision == SWKB_FP64;
    size_t smem = p->fc ? (f64 ? fc_resum_smem_bytes<double>(p->wcap, p->TM)
                               : fc_resum_smem_bytes<float>(p->wcap, p->TM))
                        : (f64 ? resum_smem_bytes<double>(p->wcap, p->TM)
                               : resum_smem_bytes<float>(p->wcap, p->TM));
    if (p->fc) smem = std::max(smem, fc_modes_smem_bytes<double>(p->fc_Np));
    if (smem > (size_t)optin)
      return fail(SWKB_ERR_INVALID_ARG, "resummation tile of %d points needs %zu B of shared "
                  "memory (%d available)", p->TM, smem, optin);
  }
  p->alloc_groups = p->n_groups;
  p->alloc_tiles = p->n_tiles;
  if (p->autotune) {
    for (const Tiling& t : tiling_candidates(p)) {
      apply_tiling(p, t);
      p->alloc_groups = std::max(p->alloc_groups, p->n_groups);
      p->alloc_tiles = std::max(p->alloc_tiles, p->n_tiles);
    }
    apply_tiling(p, def);
  }
  return SWKB_OK;
}

// Device bytes build_device will allocate for a configured plan.
size_t device_bytes(const swkb_plan* p) {
  const size_t T = p->precision == SWKB_FP64 ? 8 : 4, V = 2 * T;
  const size_t S = 2 * (size_t)p->Nt + 1;
  size_t b = (size_t)p->n_cols * (T == 8 ? (size_t)p->n_int * 8                      // medium
                                          : (size_t)table32_intervals(p) *
                                                (p->pieces > 0 ? 4 * p->pieces : 8)) * T;
  b += (size_t)p->stage_rows * S * (sizeof(int) + T);               // stage columns
  b += 3 * (size_t)p->M * T + (size_t)p->M * V;                     // mode tables
  b += (size_t)p->N * V;                                            // twiddles
  if (p->absorber_frac > 0) b += (size_t)p->N * T;                  // absorber
  b += (size_t)p->N * V * (2 + (size_t)p->alloc_groups) + (size_t)p->M * V;  // u, Y, partials, c
  if (T == 4) b += (size_t)p->M * V;                                 // polar c
  b += 3 * (size_t)p->NRT * p->Mr * T * (p->overlap ? 2 : 1);     // rays (one or two sets)
  if (p->planes > 1)                                                 // inner planes
    b += (size_t)(p->planes - 1) * (3 * (size_t)p->NRT * p->Mr * T + (size_t)p->M * V) +
         (size_t)p->M * V * (T == 4 ? 2 : 1);
  b += (size_t)(p->alloc_tiles + 1) * p->Mr * sizeof(int) * (p->sym ? 2 : 1) *
       (p->overlap ? 2 : 1);
  b += 16 + 2 * (size_t)std::max(p->N, p->n_z) * sizeof(double);   // status, io
  if (p->fc) {
    b -= (size_t)p->N * V * 2;                                       // no twiddles, no Y
    b += (size_t)FC_CONT_ROWS * FC_CONT_COLS * 8 + (size_t)p->fc_Np * 16   // operator, twiddles
         + (size_t)p->NRT * (sizeof(int) + V)                        // launch-point weights
         + (size_t)p->fc_P * p->M * V * (p->planes > 1 ? 2 : 1);     // patch coefficients
  }
  return b;
}

}  // namespace

namespace {

template <typename T>
swkb_status begin_t(swkb_plan* p, const double* u0_host) {
  using V = typename C2<T>::type;
  p->rays_ready = false;
  CK(cudaMemcpyAsync(p->io, u0_host, 2 * sizeof(double) * p->n_z, cudaMemcpyHostToDevice,
                     p->stream));
  TRY(timed(p, SWKB_KERNEL_INIT, 1,
            [&] { return launch_init<T>(p->io, p->n_z, p->fc ? p->n_z : p->N, p->mirror,
                                        (V*)p->u, p->stream); }));
  if (p->overlap) {   // both ray-buffer sets free
    CK(cudaEventRecord(p->ev_free[0], p->stream));
    CK(cudaEventRecord(p->ev_free[1], p->stream));
  }
  return SWKB_OK;
}

template <typename T>
swkb_status finish_t(swkb_plan* p, bool fresh) {
  using V = typename C2<T>::type;
  if (!fresh) TRY(reduce_to_u<T>(p, true));
  const int off = p->mirror ? p->n_z : 0;
  TRY(timed(p, SWKB_KERNEL_OUTPUT, 1,
            [&] { return launch_output<T>((const V*)p->u, off, p->n_z, p->io, p->stream); }));
  return SWKB_OK;
}

std::mutex g_tune_mutex;
std::map<std::string, Tiling> g_tune_cache;

std::string tune_key(const swkb_plan* p) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%d/%d/%d/%d/%d/%d/%d/%d/%d/%d/%d", p->precision, p->device, p->sms,
           p->N, p->M, p->Mr, p->NRT, p->R, p->Nt, p->sym, p->n_cols > 1);
  return buf;
}

// Time every candidate tiling on this plan's own buffers (two screens each,
// after one warm-up screen, CUDA events on the plan's stream) and keep the
// fastest; the choice is cached per shape for the rest of the process.
template <typename T>
swkb_status autotune_plan(swkb_plan* p) {
  Range range("swkb_autotune");
  using V = typename C2<T>::type;
  const std::string key = tune_key(p);
  {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      apply_tiling(p, it->second);
      return SWKB_OK;
    }
  }
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  CK(cudaMemsetAsync(p->u, 0, (size_t)p->N * sizeof(V), p->stream));
  CK(cudaMemsetAsync(p->part, 0, (size_t)p->alloc_groups * p->N * sizeof(V), p->stream));
  CK(cudaMemsetAsync(p->io, 0, 2 * (size_t)std::max(p->N, p->n_z) * sizeof(double), p->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  Tiling best = default_tiling(p);
  float best_ms = 1e30f;
  swkb_status st = SWKB_OK;
  for (const Tiling& t : tiling_candidates(p)) {
    apply_tiling(p, t);
    p->rays_ready = false;   // brackets depend on the tile size
    if (resum_smem_bytes<T>(p->wcap, p->TM) > (size_t)optin) continue;
    // time what a propagation runs: with rays on their own stream, four
    // overlapped screens (zero field in and out of the staging buffer);
    // otherwise two screens after a warm-up screen
    if (p->overlap) {
      st = enqueue_overlapped<T>(p, p->io, 0, 1, p->io, nullptr, 0);
    } else {
      st = launch_screen<T>(p, 0, true);
    }
    if (st != SWKB_OK) break;
    float ms = 1e30f;
    for (int trial = 0; trial < 3 && st == SWKB_OK; ++trial) {   // min of 3 trials
      cudaEventRecord(e0, p->stream);
      if (p->overlap) {
        st = enqueue_overlapped<T>(p, p->io, 0, 4, p->io, nullptr, 0);
      } else {
        for (int r = 1; r <= 2 && st == SWKB_OK; ++r) st = launch_screen<T>(p, r, false);
      }
      if (st != SWKB_OK) break;
      cudaEventRecord(e1, p->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e != cudaSuccess) {
        st = fail(SWKB_ERR_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
        break;
      }
      ms = std::min(ms, t);
    }
    if (st != SWKB_OK) break;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  apply_tiling(p, best);
  CK(cudaMemsetAsync(p->status, 0, sizeof(unsigned), p->stream));
  CK(cudaStreamSynchronize(p->stream));
  memset(&p->stats, 0, sizeof(p->stats));
  if (st != SWKB_OK) return st;
  std::lock_guard<std::mutex> lk(g_tune_mutex);
  g_tune_cache[key] = best;
  return SWKB_OK;
}

}  // namespace

namespace swkb {

template <typename T>
swkb_status plan_parts(swkb_plan* p, PlanParts<T>* o) {
  using V = typename C2<T>::type;
  if ((p->precision == SWKB_FP64) != (sizeof(T) == 8))
    return fail(SWKB_ERR_INVALID_ARG, "plan precision does not match the batch");
  if (p->planes > 1 || p->reuse_rays)
    return fail(SWKB_ERR_INVALID_ARG, "batched plans march every screen and have no inner planes");
  if (p->fc) return fail(SWKB_ERR_INVALID_ARG, "the batch kernel runs periodic and grounded plans");
  if (p->N1 < 2)
    return fail(SWKB_ERR_INVALID_ARG, "batched plans need a two-pass DFT (fft_n1 >= 2)");
  *o = PlanParts<T>{};
  o->N = p->N; o->n_z = p->n_z; o->M = p->M; o->Mr = p->Mr; o->NRT = p->NRT; o->Nt = p->Nt;
  o->n_max = p->n_max; o->mirror = p->mirror; o->sym = p->sym; o->N1 = p->N1;
  o->n_cols = p->n_cols; o->pieces = p->pieces;
  o->stage_rows = p->stage_rows;
  o->stage_stride = 2 * p->Nt + 1;
  if (sizeof(T) == 8) {
    o->march_bx = (p->Mr + 31) / 32;
    o->march_blocks = o->march_bx * ((p->NRT + 7) / 8);
  } else {
    o->march_bx = 0;
    o->march_blocks = (int)(((long long)p->Mr * ((p->NRT + 1) / 2) + 255) / 256);
  }
  o->bracket_bx = (p->Mr + 255) / 256;
  o->resum_blocks = p->n_tiles_run * p->n_groups;
  o->resum_pw = p->PW;
  o->resum_smem = resum_smem_bytes<T>(p->wcap, p->TM);
  o->fft1_blocks = p->N2 / FFT1_COLS;
  o->fft2_blocks = p->mirror ? p->n_max + 1 : p->M;
  o->fft1_smem = fft1_smem_bytes<T>(p->N1);
  o->reduce_n = (p->mirror || p->sym) ? p->N / 2 + 1 : p->N;
  o->out_off = p->mirror ? p->n_z : 0;
  o->rays = (size_t)p->NRT * p->Mr;
  o->jlo_n = (size_t)(p->alloc_tiles + 1) * p->Mr;
  o->sets = p->overlap ? 2 : 1;
  o->rd[0] = (T*)p->rd; o->rph[0] = (T*)p->rph; o->ra[0] = (T*)p->ra;
  o->jlo[0] = p->jlo; o->jneg[0] = p->jlo_neg;
  o->rd[1] = (T*)p->rd1; o->rph[1] = (T*)p->rph1; o->ra[1] = (T*)p->ra1;
  o->jlo[1] = p->jlo1; o->jneg[1] = p->jlo_neg1;
  o->u = (V*)p->u;
  o->status = p->status;
  o->fft_fresh = fft_args<T>(p, false);
  o->fft_next = fft_args<T>(p, true);
  o->fin = ReduceArgs<T>{(const V*)p->part, p->n_groups, p->N, (const T*)p->W, p->mirror, p->sym,
                         (V*)p->u};
  o->march = march_args<T>(p, 0);
  o->bracket = bracket_args<T>(p, (const T*)p->rd);
  o->resum = resum_args<T>(p, (const T*)p->rd, (const T*)p->rph, (const T*)p->ra,
                           (const V*)p->c);
  return SWKB_OK;
}
template swkb_status plan_parts<float>(swkb_plan*, PlanParts<float>*);
template swkb_status plan_parts<double>(swkb_plan*, PlanParts<double>*);

cudaStream_t plan_stream(swkb_plan* p) { return p->stream; }
size_t plan_bytes(const swkb_plan* p) { return p->bytes; }

swkb_status plan_begin(swkb_plan* p, const double* u0_host) {
  CK(cudaSetDevice(p->device));
  return p->precision == SWKB_FP64 ? begin_t<double>(p, u0_host) : begin_t<float>(p, u0_host);
}

swkb_status plan_advance(swkb_plan* p, int q, int n, bool first) {
  CK(cudaSetDevice(p->device));
  // with rays on their own stream, screens alternate between the two ray-buffer
  // sets by the parity of their index
  for (int i = 0; i < n; ++i) {
    const bool fresh = first && i == 0;
    const int qi = q + i;
    swkb_status st;
    if (p->overlap)
      st = p->precision == SWKB_FP64 ? overlapped_screen<double>(p, qi, qi & 1, fresh)
                                     : overlapped_screen<float>(p, qi, qi & 1, fresh);
    else
      st = p->precision == SWKB_FP64 ? launch_screen<double>(p, qi, fresh)
                                     : launch_screen<float>(p, qi, fresh);
    if (st != SWKB_OK) return st;
  }
  return SWKB_OK;
}

swkb_status plan_finish(swkb_plan* p, bool fresh) {
  CK(cudaSetDevice(p->device));
  return p->precision == SWKB_FP64 ? finish_t<double>(p, fresh) : finish_t<float>(p, fresh);
}

swkb_status plan_collect(swkb_plan* p, double* out_host) {
  CK(cudaSetDevice(p->device));
  swkb_status st = read_status(p);   // synchronises the plan's stream
  if (st != SWKB_OK) return st;
  CK(cudaMemcpy(out_host, p->io, 2 * sizeof(double) * p->n_z, cudaMemcpyDeviceToHost));
  return SWKB_OK;
}

swkb_status estimate_plan_bytes(const swkb_profile* prof, double k, const swkb_domain* dom,
                                int32_t n_z, double screen_dx, const swkb_options* opt_in,
                                size_t* bytes) {
  try {
    swkb_options opt;
    if (opt_in) opt = *opt_in; else swkb_options_default(&opt);
    swkb_plan tmp;
    TRY(configure(&tmp, prof, k, dom, n_z, screen_dx, opt));
    *bytes = device_bytes(&tmp);
    return SWKB_OK;
  } catch (...) {
    return fail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

}  // namespace swkb

extern "C" {

swkb_status swkb_plan_create(const swkb_profile* prof, double k, const swkb_domain* dom,
                             int32_t n_z, double screen_dx, const swkb_options* opt_in,
                             swkb_plan** out) {
  Range range("swkb_plan_create");
  try {
    if (!out) return fail(SWKB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    swkb_options opt;
    if (opt_in) opt = *opt_in; else swkb_options_default(&opt);
    swkb_plan* p = new swkb_plan();
    struct Guard { swkb_plan*& p; ~Guard() { if (p) release(p); } } guard{p};
    TRY(configure(p, prof, k, dom, n_z, screen_dx, opt));
    const char* ge = getenv("SWKB_GRAPHS");
    p->use_graphs = !(ge && ge[0] == '0');
    const char* fe = getenv("SWKB_FUSE_REDUCE");
    p->fuse_reduce = !(fe && fe[0] == '0');
    if (opt.cuda_stream) {
      p->stream = (cudaStream_t)opt.cuda_stream;
    } else {
      CK(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
      p->own_stream = true;
    }
    if (p->overlap) {
      CK(cudaStreamCreateWithFlags(&p->ray_stream, cudaStreamNonBlocking));
      for (int b = 0; b < 2; ++b) {
        CK(cudaEventCreateWithFlags(&p->ev_rays[b], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&p->ev_free[b], cudaEventDisableTiming));
      }
    }
    swkb_status st = p->precision == SWKB_FP64 ? build_device<double>(p, prof)
                                               : build_device<float>(p, prof);
    if (st != SWKB_OK) return st;
    if (p->autotune) {
      st = p->precision == SWKB_FP64 ? autotune_plan<double>(p) : autotune_plan<float>(p);
      if (st != SWKB_OK) return st;
    }
    CK(cudaStreamSynchronize(p->stream));
    *out = p;
    p = nullptr;  // disarm guard
    return SWKB_OK;
  } catch (const std::exception& e) {
    return fail(SWKB_ERR_OOM, "host allocation failed: %s", e.what());
  } catch (...) {
    return fail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

swkb_status swkb_plan_get_info(const swkb_plan* p, swkb_plan_info* info) {
  if (!p || !info) return fail(SWKB_ERR_INVALID_ARG, "NULL argument");
  info->n_fft = p->N;
  info->n_max = p->n_max;
  info->n_modes = p->M;
  info->n_rays = p->N_r;
  info->n_ghost = p->G;
  info->n_rays_total = p->NRT;
  info->tile_points = p->TM;
  info->mode_groups = p->n_groups;
  info->march_modes = p->Mr;
  info->resum_points = p->n_tiles_run * p->TM;
  info->fft_n1 = p->N1;
  info->dz = p->dz;
  info->period = p->L;
  info->eps_ref = p->eps_ref;
  info->device_bytes = p->bytes;
  info->medium_pieces = p->pieces;
  info->ctas_per_sm = p->ctas_per_sm;
  info->fc_patches = p->fc_P;
  info->fc_period_points = p->fc_Np;
  return SWKB_OK;
}

swkb_status swkb_propagate(swkb_plan* p, const double* u0, int32_t q0, int32_t n_screens,
                           double* u_out, int32_t snapshot_every, int32_t on_device) {
  Range range("swkb_propagate");
  try {
    if (!p || !u0 || !u_out) return fail(SWKB_ERR_INVALID_ARG, "NULL argument");
    if (n_screens < 0 || q0 < 0) return fail(SWKB_ERR_INVALID_ARG, "negative screen count");
    if (snapshot_every < 0 || (snapshot_every > 0 && n_screens % snapshot_every))
      return fail(SWKB_ERR_INVALID_ARG, "snapshot_every must divide n_screens");
    CK(cudaSetDevice(p->device));
    const size_t nb = 2 * sizeof(double) * p->n_z;
    if (n_screens == 0) {
      if (on_device) CK(cudaMemcpyAsync(u_out, u0, nb, cudaMemcpyDeviceToDevice, p->stream));
      else memcpy(u_out, u0, nb);
      if (on_device) CK(cudaStreamSynchronize(p->stream));
      return SWKB_OK;
    }
    const double* din = u0;
    if (!on_device) {
      CK(cudaMemcpyAsync(p->io, u0, nb, cudaMemcpyHostToDevice, p->stream));
      din = p->io;   // consumed by the init kernel before any output reuses io
    }
    double* odev = on_device ? u_out : nullptr;
    double* ohost = on_device ? nullptr : u_out;
    return p->precision == SWKB_FP64
               ? run<double>(p, din, q0, n_screens, odev, ohost, snapshot_every)
               : run<float>(p, din, q0, n_screens, odev, ohost, snapshot_every);
  } catch (...) {
    return fail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

swkb_status swkb_propagate_planes(swkb_plan* p, const double* u0, int32_t q0, int32_t n_screens,
                                  int32_t planes, double* u_out, int32_t on_device) {
  Range range("swkb_propagate_planes");
  try {
    if (!p || !u0 || !u_out) return fail(SWKB_ERR_INVALID_ARG, "NULL argument");
    if (n_screens < 0 || q0 < 0) return fail(SWKB_ERR_INVALID_ARG, "negative screen count");
    if (planes < 1 || p->Nt % planes)
      return fail(SWKB_ERR_INVALID_ARG, "planes (%d) must divide rk4_steps (%d)", planes, p->Nt);
    if (planes > std::max(1, p->planes))
      return fail(SWKB_ERR_INVALID_ARG,
                  "plan holds buffers for %d planes per screen (swkb_options.planes)",
                  std::max(1, p->planes));
    CK(cudaSetDevice(p->device));
    if (n_screens == 0) return SWKB_OK;
    const bool f64 = p->precision == SWKB_FP64;
    if (planes > 1) TRY(f64 ? upload_plane_phases<double>(p, planes)
                            : upload_plane_phases<float>(p, planes));
    const size_t nb = 2 * sizeof(double) * p->n_z;
    const double* din = u0;
    if (!on_device) {
      CK(cudaMemcpyAsync(p->io, u0, nb, cudaMemcpyHostToDevice, p->stream));
      din = p->io;   // consumed by the init kernel before any output reuses io
    }
    double* odev = on_device ? u_out : nullptr;
    double* ohost = on_device ? nullptr : u_out;
    TRY(f64 ? enqueue_planes<double>(p, din, q0, n_screens, planes, odev, ohost)
            : enqueue_planes<float>(p, din, q0, n_screens, planes, odev, ohost));
    return read_status(p);
  } catch (...) {
    return fail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

swkb_status swkb_debug_screen(swkb_plan* p, int32_t q, const double* u_full, double* c,
                              double* delta, double* r, double* a, double* u_next) {
  try {
    if (!p || !u_full) return fail(SWKB_ERR_INVALID_ARG, "NULL argument");
    if (p->fc) return fail(SWKB_ERR_INVALID_ARG, "patch-wise plans have no single mode set");
    CK(cudaSetDevice(p->device));
    return p->precision == SWKB_FP64 ? debug_screen<double>(p, q, u_full, c, delta, r, a, u_next)
                                     : debug_screen<float>(p, q, u_full, c, delta, r, a, u_next);
  } catch (...) {
    return fail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

void swkb_plan_destroy(swkb_plan* p) { release(p); }

swkb_status swkb_plan_set_timing(swkb_plan* p, int32_t kinds, int32_t every) {
  if (!p) return fail(SWKB_ERR_INVALID_ARG, "NULL plan");
  if (every < 1) return fail(SWKB_ERR_INVALID_ARG, "every must be >= 1");
  p->timing = (unsigned)kinds & ((1u << SWKB_KERNEL_KINDS) - 1u);
  p->timing_serial = p->timing != 0 && (kinds & SWKB_TIME_SERIAL) != 0;
  p->timing_every = every;
  memset(p->timing_seen, 0, sizeof(p->timing_seen));
  p->marks.clear();
  memset(&p->stats, 0, sizeof(p->stats));
  return SWKB_OK;
}

swkb_status swkb_plan_get_stats(const swkb_plan* p, swkb_plan_stats* st) {
  if (!p || !st) return fail(SWKB_ERR_INVALID_ARG, "NULL argument");
  *st = p->stats;
  return SWKB_OK;
}

}  // extern "C"
