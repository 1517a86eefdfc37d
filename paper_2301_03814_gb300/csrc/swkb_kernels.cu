// Device kernels of the screened-WKB screen step (sm_103a), templated on the
// arithmetic type T (double: the FP64 path; float: the mixed path, whose
// FP64 parts -- the range-phase carry exp(i Phi_n) and the launch tables --
// are prepared on the host).
//
// One screen Gamma_q -> Gamma_{q+1} (Algorithm 1) is, on the device:
//   k_reduce   sum the resummation partials, absorber window, reflection
//              projection u <- (u(z) +- u(2 z_a - z)) / 2   (Sec. 2.3)
//   k_fft1/2   pruned DFT of the screen field, c_n = w_n / N * exp(i Phi_n)
//              for |n| <= n_max                        (Eqs. fft_eq, ifft_eq)
//   k_march    RK4 across the slab for every (mode, ray): the x-form of the
//              characteristic system and its s-variation (Eqs. charsys,
//              charsys_s), amplitude sqrt(P0 / (P1 Z_s)) (corrected Eq.
//              delta_psi_eq_jac)
//   k_bracket  landing monotonicity / coverage checks, first bracket ray of
//              every resummation tile
//   k_resum    4-point Lagrange interpolation of phase and amplitude onto the
//              grid (Eq. ray_bundle_q_plus_1) fused with the modal sum
//
// The ray state is marched as deviations from the launch values:
//   dz = z - s,  dQ = Q - kappa_n,  rh = r - x P_bar_n,
// with P_bar_n = sqrt(eps_ref - kappa_n^2) and the table storing
// eps - eps_ref.  In exact arithmetic this is the same ODE as the plain form
// (RK4 is invariant under adding a constant to one right-hand side), but
// every stored quantity is small, so FP32 keeps ~1e-7 of the *deviation*.
// The dropped constant x P_bar_n is restored on the host, in FP64 and reduced
// mod 2 pi, as exp(i k dx P_bar_n) folded into c_n.

#include <utility>

#include "swkb_device.cuh"

namespace swkb {

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
namespace {
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args&&... args) {
  k<<<grid, block, smem, s>>>(std::forward<Args>(args)...);
  return cudaGetLastError();
}
}  // namespace

template <typename T>
cudaError_t launch_init(const double* u0, int n_z, int N, int mirror, typename C2<T>::type* u,
                        cudaStream_t s) {
  return launch_k(k_init<T>, dim3((N + 255) / 256), dim3(256), 0, s, u0, n_z, N, mirror, u);
}

template <typename T>
cudaError_t launch_reduce(const ReduceArgs<T>& a, cudaStream_t s) {
  const int n = (a.mirror || a.sym) ? a.N / 2 + 1 : a.N;
  return launch_k(k_reduce<T>, dim3((n + 255) / 256), dim3(256), 0, s, a);
}

template <typename T>
size_t fft1_smem_bytes(int N1) {
  return (size_t)(N1 * FFT1_COLS + N1) * sizeof(typename C2<T>::type);
}

template <typename T>
cudaError_t launch_fft(const FftArgs<T>& a, cudaStream_t s) {
  if (a.N1 > 1) {
    const size_t smem = fft1_smem_bytes<T>(a.N1);
    const cudaError_t e = launch_k(k_fft1<T>, dim3(a.N2 / FFT1_COLS), dim3(256), smem, s, a);
    if (e != cudaSuccess) return e;
  }
  const int modes = a.mirror ? a.n_max + 1 : 2 * a.n_max + 1;
  return launch_k(k_fft2<T>, dim3(modes), dim3(FFT2_THREADS), 0, s, a);
}

template <typename T>
cudaError_t launch_march(const MarchArgs<T>& a, bool multi_column, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.Mr + 31) / 32, (a.NRT + 7) / 8);
  if (a.plane_steps > 0)
    return multi_column ? launch_k(k_march<T, true, true>, grid, block, 0, s, a)
                        : launch_k(k_march<T, false, true>, grid, block, 0, s, a);
  return multi_column ? launch_k(k_march<T, true, false>, grid, block, 0, s, a)
                      : launch_k(k_march<T, false, false>, grid, block, 0, s, a);
}

template <>
cudaError_t launch_march<float>(const MarchArgs<float>& a, bool multi_column, cudaStream_t s) {
  const long long threads = (long long)a.Mr * ((a.NRT + 1) / 2);
  const dim3 block(256), grid((unsigned)((threads + 255) / 256));
  const bool pl = a.plane_steps > 0, cub = a.med.pieces > 0;
  if (cub) {
    if (pl)
      return multi_column ? launch_k(k_march_x2<true, true, true>, grid, block, 0, s, a)
                          : launch_k(k_march_x2<false, true, true>, grid, block, 0, s, a);
    return multi_column ? launch_k(k_march_x2<true, false, true>, grid, block, 0, s, a)
                        : launch_k(k_march_x2<false, false, true>, grid, block, 0, s, a);
  }
  if (pl)
    return multi_column ? launch_k(k_march_x2<true, true, false>, grid, block, 0, s, a)
                        : launch_k(k_march_x2<false, true, false>, grid, block, 0, s, a);
  return multi_column ? launch_k(k_march_x2<true, false, false>, grid, block, 0, s, a)
                      : launch_k(k_march_x2<false, false, false>, grid, block, 0, s, a);
}

template <typename T>
cudaError_t launch_bracket(const BracketArgs<T>& a, cudaStream_t s) {
  const int rows = (a.NRT - 1 + BRACKET_RUN - 1) / BRACKET_RUN;
  dim3 grid((a.Mr + 255) / 256, rows < 65535 ? rows : 65535);
  return launch_k(k_bracket<T>, grid, dim3(256), 0, s, a);
}

template <typename T>
size_t resum_smem_bytes(int wcap, int tile_points) {
  const size_t per_warp = ((RESUM_CF + 3) * (size_t)wcap * sizeof(T) + 15) & ~(size_t)15;
  const size_t stage = (size_t)RESUM_WARPS * per_warp;
  // 32 runs of PW points, each padded to PW + 1 entries
  const size_t red = (size_t)RESUM_WARPS * (tile_points + 32) * sizeof(typename C2<T>::type);
  return stage > red ? stage : red;
}

template <typename T>
cudaError_t launch_resum(const ResumArgs<T>& a, cudaStream_t s) {
  const int grid = a.n_tiles_run * a.n_groups;
  const size_t smem = resum_smem_bytes<T>(a.wcap, a.TM);
  const int threads = RESUM_WARPS * 32;
  switch (a.PW) {
    case 2: return launch_k(k_resum<T, 2>, dim3(grid), dim3(threads), smem, s, a);
    case 4: return launch_k(k_resum<T, 4>, dim3(grid), dim3(threads), smem, s, a);
    case 8: return launch_k(k_resum<T, 8>, dim3(grid), dim3(threads), smem, s, a);
    case 16: return launch_k(k_resum<T, 16>, dim3(grid), dim3(threads), smem, s, a);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t prepare_kernels(int resum_smem) {
  // The limit is a per-device property of the kernel shared by every plan in
  // the process: raise it to the device's opt-in maximum (never lower it, or
  // a plan with smaller tiles would break another plan's launches).
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (resum_smem > optin) return cudaErrorInvalidValue;
  const void* fs[] = {(const void*)k_resum<T, 2>, (const void*)k_resum<T, 4>,
                      (const void*)k_resum<T, 8>, (const void*)k_resum<T, 16>};
  for (const void* f : fs) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t prepare_fft_kernels() {
  // k_fft1's dynamic shared memory is (N1 FFT1_COLS + N1) complex values: at
  // most 9 KB for the largest split the plans allow (N1 = 64), inside the
  // default 48 KB limit; k_fft2 uses static shared memory only
  static_assert((64 * FFT1_COLS + 64) * 16 <= 48 * 1024, "k_fft1 staging exceeds 48 KB");
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_cscale(const typename C2<T>::type* c, const typename C2<T>::type* f,
                          typename C2<T>::type* out, typename C2<T>::type* pol, int M,
                          cudaStream_t s) {
  return launch_k(k_cscale<T>, dim3((M + 255) / 256), dim3(256), 0, s, c, f, out, pol, M);
}

template <typename T>
cudaError_t launch_output(const typename C2<T>::type* u, int offset, int n, double* out,
                          cudaStream_t s) {
  return launch_k(k_output<T>, dim3((n + 255) / 256), dim3(256), 0, s, u, offset, n, out);
}

#define SWKB_INSTANTIATE(T)                                                                     \
  template cudaError_t launch_init<T>(const double*, int, int, int, C2<T>::type*, cudaStream_t); \
  template cudaError_t launch_reduce<T>(const ReduceArgs<T>&, cudaStream_t);                    \
  template cudaError_t launch_fft<T>(const FftArgs<T>&, cudaStream_t);                          \
  template cudaError_t launch_march<T>(const MarchArgs<T>&, bool, cudaStream_t);                \
  template cudaError_t launch_bracket<T>(const BracketArgs<T>&, cudaStream_t);                  \
  template cudaError_t launch_resum<T>(const ResumArgs<T>&, cudaStream_t);                      \
  template cudaError_t launch_output<T>(const C2<T>::type*, int, int, double*, cudaStream_t);   \
  template cudaError_t launch_cscale<T>(const C2<T>::type*, const C2<T>::type*, C2<T>::type*,   \
                                        C2<T>::type*, int, cudaStream_t);                       \
  template size_t resum_smem_bytes<T>(int, int);                                                \
  template size_t fft1_smem_bytes<T>(int);                                                      \
  template cudaError_t prepare_kernels<T>(int);                                                 \
  template cudaError_t prepare_fft_kernels<T>();

SWKB_INSTANTIATE(float)
SWKB_INSTANTIATE(double)

}  // namespace swkb
