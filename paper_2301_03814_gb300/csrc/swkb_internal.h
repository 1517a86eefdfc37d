// Internal declarations shared by the kernel and host translation units of
// libswkb.so.  Nothing here is part of the public C ABI (include/swkb.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "swkb.h"

namespace swkb {

// Status bits written by device code (atomicOr) and mapped to swkb_status.
enum : unsigned {
  ST_CAUSTIC = 1u,   // Z_s <= 0 or landings not increasing
  ST_TURNING = 2u,   // eps - Q^2 <= 0
  ST_RANGE = 4u,     // left the permittivity table
  ST_COVER = 8u,     // ghost rays do not cover the screen
  ST_BOUNDS = 16u,   // bounds-checked builds: a device index left its buffer
};

// Columns n2 of the DFT's pass 1 handled by one block.
constexpr int FFT1_COLS = 8;

template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

// Quintic medium table: per column, per z interval i, the monomial
// coefficients a0..a5 of eps(z0 + (i + t) h) - eps_ref in t in [0, 1]
// (8 slots per interval, the last two unused).
//   FP64 plans: the profile's n_int intervals from z0 = z_a; grounded domains
//   reflect z about z_mirror before the lookup.
//   FP32 plans: the reflection is stored instead (grounded domains: the
//   mirror images of the n_int intervals below z_a, then the n_int intervals
//   above), followed by one interval continuing the last one, so that a
//   position exactly at the top has a t = 0 entry; n_int counts the intervals
//   before that pad and top = n_int as a float.  When pieces = S > 0 every
//   interval is stored as S cubic Hermite pieces of its quintic (value and
//   slope matched at the piece ends; 4 slots b0..b3 in the piece's own
//   tau in [0, 1]) and n_int, top, inv_h, inv_h2 count pieces.
template <typename T>
struct Medium {
  const T* coef;
  int n_int;
  long long col_stride;
  T z0, inv_h, inv_h2;
  int mirrored;
  T z_mirror;
  T top;
  int pieces;   // FP32: > 0 when each entry is a cubic piece (4 slots), in piece units
  long long size;   // values in coef (all columns), for bounds-checked builds
};

// Per-screen RK4 stage columns: stage l = 0 .. 2 N_t sits at x_q + l h / 2;
// eps there is (1 - th) col[c] + th col[c + 1].
template <typename T>
struct Stages {
  const int* c;
  const T* th;
};

template <typename T>
struct MarchArgs {
  Medium<T> med;
  Stages<T> st;
  const T* kappa;   // [M] kappa_n
  const T* pbar;    // [M] sqrt(eps_ref - kappa_n^2)
  const T* pbar2;   // [M] eps_ref - kappa_n^2
  int Mr;           // marched modes (row length of the outputs)
  int mode_off;     // marched mode r is mode index r + mode_off (n = r + mode_off - n_max)
  int NRT, G, R, Nt;
  T z_lo, dz, inv_dz, h, k_over_2pi;
  T u_lo, u_dz;     // FP32 table position of grid point 0 and per grid point
  T* out_d;         // [NRT][Mr] landing offset from the launch grid point, grid units
  T* out_ph;        // [NRT][Mr] residual phase k (r - x P_bar) / (2 pi), turns
  T* out_a;         // [NRT][Mr] amplitude factor sqrt(P0 / (P1 Z_s))
  // fields between screens: after every plane_steps RK4 steps (before the
  // last) the same three quantities go to plane j = steps / plane_steps - 1
  // of pl_d / pl_ph / pl_a, [planes - 1][NRT][Mr]; plane_steps = 0: none
  int plane_steps;
  T* pl_d;
  T* pl_ph;
  T* pl_a;
  unsigned* status;
};

template <typename T>
struct BracketArgs {
  const T* d;       // [NRT][Mr]
  int Mr, NRT, G, R, N, TM, n_tiles;
  int* jlo;         // [n_tiles + 1][Mr] bracket ray of each tile start
  int sym;          // grounded domain: also the mirrored family of each mode
  int* jlo_neg;     // [n_tiles + 1][Mr] brackets of the mirror image (mode -n)
  unsigned* status;
};

template <typename T>
struct ResumArgs {
  const T* d;
  const T* ph;
  const T* a;
  const int* jlo;
  const int* jlo_neg;
  const typename C2<T>::type* c;   // [M] mode coefficients, range phase folded in
  const typename C2<T>::type* cpol; // [M] FP32: (|c_n|, arg(c_n) / 2 pi), read instead of c
  int M, Mr, NRT, G, R, N, TM, PW, n_tiles, n_groups, modes_per_group, n_max, wcap;
  int sym;          // grounded: modes n < 0 are mirror images of -n; only the
                    // tiles of the physical half and tile 0 are summed
  int n_tiles_run;  // tiles summed per mode group
  typename C2<T>::type* part;      // [n_groups][N], one partial sum per mode group
  unsigned* status;
};

template <typename T>
struct ReduceArgs {
  const typename C2<T>::type* part;  // [n_part][N]
  int n_part, N;
  const T* W;                        // [N] absorber or nullptr
  int mirror;                        // 0 none, +1 even, -1 odd
  int sym;                           // partials cover only m >= N/2 and m = 0
  typename C2<T>::type* u;           // [N]
};

template <typename T>
struct FftArgs {
  const typename C2<T>::type* u;     // [N]
  const typename C2<T>::type* tw;    // [N] exp(-2 pi i k / N)
  typename C2<T>::type* Y;           // [N1][N2]
  int N, N1, N2, log2N2, n_max;
  int mirror;                        // 0, or +-1: the field is even / odd
  // pass 1 may form the field itself from the resummation partials (absorber
  // and reflection as in ReduceArgs) instead of reading u
  const typename C2<T>::type* part;  // [n_part][N] or nullptr: read u
  int n_part, sym;
  const T* W;
  T inv_N;
  const typename C2<T>::type* ephi;  // [M] exp(i Phi_n)
  typename C2<T>::type* c;           // [M]
  typename C2<T>::type* cpol;        // [M] (|c_n|, arg(c_n) / 2 pi), or nullptr
};

// Patch-wise Fourier-continuation screens (swkb_fc.cu).  Patch p holds the
// grid points p stride .. p stride + n_pat - 1 of the non-periodic interval.
template <typename T>
struct FcModesArgs {
  const typename C2<T>::type* u;     // [>= n_z] the screen field
  int n_pat, stride, P, Np, n_max, M;
  const double* cont;                // [FC_C][FC_D] continuation operator
  const double2* tw;                 // [Np] exp(-2 pi i k / Np)
  const typename C2<T>::type* ephi;  // [M] exp(i k dx Pbar_n)
  double inv_Np;
  unsigned np_magic;                 // floor(2^32 / Np)
  typename C2<T>::type* cf;          // [P][M] out: rotated, carried mode coefficients
};

template <typename T>
struct FcResumArgs {
  const T* d;                        // [NRT][M] rays, as for the periodic resummation
  const T* ph;
  const T* a;
  const int* jlo;                    // [n_tiles + 1][M]
  const typename C2<T>::type* cf;    // [P][M]
  const int* win_p;                  // [NRT] first patch with a non-zero weight at ray j
  const typename C2<T>::type* win_s; // [NRT] (S^{p0}, S^{p0+1}) at ray j
  int M, NRT, G, R, N, TM, n_tiles, n_groups, modes_per_group, n_max, wcap, Np, P;
  unsigned np_magic;                 // floor(2^32 / Np)
  typename C2<T>::type* part;        // [n_groups][N]
  unsigned* status;
};

template <typename T> cudaError_t launch_fc_modes(const FcModesArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_fc_resum(const FcResumArgs<T>& a, cudaStream_t s);
// out[p][n] = cf[p][n] f[n] for P patches of M modes (planes inside a screen)
template <typename T> cudaError_t launch_fc_cscale(const typename C2<T>::type* cf,
                                                   const typename C2<T>::type* f,
                                                   typename C2<T>::type* out, int P, int M,
                                                   cudaStream_t s);
template <typename T> size_t fc_resum_smem_bytes(int wcap, int tile_points);
template <typename T> size_t fc_modes_smem_bytes(int Np);
template <typename T> cudaError_t prepare_fc_kernels(int resum_smem, int modes_smem);
// The FC-Gram continuation operator ([FC_C][FC_D], row-major) and its sizes.
const double* fc_continuation_host();
constexpr int FC_CONT_ROWS = 25, FC_CONT_COLS = 5;

// launchers (defined in swkb_kernels.cu for T = float, double)
template <typename T> cudaError_t launch_init(const double* u0, int n_z, int N, int mirror,
                                              typename C2<T>::type* u, cudaStream_t s);
template <typename T> cudaError_t launch_reduce(const ReduceArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_fft(const FftArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_march(const MarchArgs<T>& a, bool multi_column,
                                               cudaStream_t s);
template <typename T> cudaError_t launch_bracket(const BracketArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_resum(const ResumArgs<T>& a, cudaStream_t s);
template <typename T> cudaError_t launch_output(const typename C2<T>::type* u, int offset, int n,
                                                double* out, cudaStream_t s);
template <typename T> cudaError_t launch_cscale(const typename C2<T>::type* c,
                                                const typename C2<T>::type* f,
                                                typename C2<T>::type* out,
                                                typename C2<T>::type* pol, int M,
                                                cudaStream_t s);
template <typename T> size_t resum_smem_bytes(int wcap, int tile_points);
// Raise the dynamic shared-memory limit of the resummation kernels
// on the current device (call once per device before launching).
template <typename T> cudaError_t prepare_kernels(int resum_smem);
// Message returned by swkb_last_error() on this thread.
void set_last_error(const char* msg);
// swkb_status of a kernel status word (ST_* bits; SWKB_OK for 0), setting
// the thread's last-error message.
swkb_status status_from_bits(unsigned bits);
// Raise only the FFT kernel's shared-memory limit on the current device.
template <typename T> cudaError_t prepare_fft_kernels();

// What the persistent batch kernel (swkb_batch.cu) takes from a plan: sizes,
// the plan's own buffers and ray-buffer sets, and the argument blocks of its
// screen steps (built exactly as the plan's own launches build them).
template <typename T>
struct PlanParts {
  int N, n_z, M, Mr, NRT, Nt, n_max, mirror, sym, N1, n_cols, pieces;
  int stage_rows, stage_stride;      // RK4 stage rows (screens q >= rows - 1 share the last)
  int march_bx, march_blocks;        // FP64: ceil(Mr / 32) x ceil(NRT / 8) blocks of (32, 8);
                                     // FP32: ceil(Mr ceil(NRT / 2) / 256) blocks of 256
  int bracket_bx;                    // bracket blocks of 256 threads along the modes
  int resum_blocks, resum_pw;        // resummation blocks (tiles x mode groups), points per lane
  size_t resum_smem;                 // shared memory of one resummation block
  int fft1_blocks, fft2_blocks;      // pass-1 blocks (N2 / FFT1_COLS), pass-2 blocks (modes formed)
  size_t fft1_smem;
  int reduce_n;                      // threads of the final reduction
  int out_off;                       // first physical point in the period
  size_t rays, jlo_n;                // values per ray array / per bracket table
  int sets;                          // ray-buffer sets the plan holds (1 or 2)
  T* rd[2];
  T* rph[2];
  T* ra[2];
  int* jlo[2];
  int* jneg[2];
  typename C2<T>::type* u;
  unsigned* status;
  FftArgs<T> fft_fresh;              // first screen: the DFT reads u
  FftArgs<T> fft_next;               // later screens: pass 1 forms u from the partials
  ReduceArgs<T> fin;                 // final reduction (projection, absorber) into u
  MarchArgs<T> march;                // screen 0's stage row, ray set 0
  BracketArgs<T> bracket;            // ray set 0
  ResumArgs<T> resum;                // ray set 0
};
// Fails (SWKB_ERR_INVALID_ARG) for plans the batch kernel does not run:
// inner planes, reused rays, or a one-pass DFT (fft_n1 = 1).
template <typename T> swkb_status plan_parts(swkb_plan* p, PlanParts<T>* out);
// Shared-memory bytes of one pass-1 DFT block for split N1.
template <typename T> size_t fft1_smem_bytes(int N1);

// Plan-level hooks used by the request server (swkb_server.cu).
cudaStream_t plan_stream(swkb_plan* p);
size_t plan_bytes(const swkb_plan* p);
// Copy the n_z-point host field in and extend it to the period (async).
swkb_status plan_begin(swkb_plan* p, const double* u0_host);
// Enqueue screens q .. q + n - 1; first: the field was just set by plan_begin.
swkb_status plan_advance(swkb_plan* p, int q, int n, bool first);
// Enqueue the final reduction and the conversion to n_z complex128 (async).
swkb_status plan_finish(swkb_plan* p, bool fresh);
// Wait for the plan's stream, map its status, copy the result to the host.
swkb_status plan_collect(swkb_plan* p, double* out_host);
// Device bytes a plan with these arguments would hold (no allocation).
swkb_status estimate_plan_bytes(const swkb_profile* prof, double k, const swkb_domain* dom,
                                int32_t n_z, double screen_dx, const swkb_options* opt,
                                size_t* bytes);

}  // namespace swkb
