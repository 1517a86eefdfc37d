// swkb_modes_noalloc: step (a) of the screen step -- the pruned DFT of one
// screen field into its kept plane-wave coefficients -- for callers that must
// not allocate device memory.
//
// Who needs it: code that owns every byte of device memory itself (a host
// framework that pre-partitions HBM and forbids other allocators, or a
// latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device and stall other streams).  Such callers still hand in their input
// and output buffers; the FFT's working storage lives here instead, in
// file-scope device arrays of a fixed size that every GPU loading this library
// holds until the process exits (3 MB per device).
//
// The arithmetic is the library's FP64 pruned two-pass DFT (k_fft1 / k_fft2),
// unchanged; only where its scratch comes from differs.

#include <mutex>
#include <string>

#include "swkb.h"
#include "swkb_internal.h"

namespace {

constexpr int kMaxN = 65536;   // largest FFT length accepted

// Scratch shared by every call on a device.  In host code these names are
// host-side stand-ins, not device addresses: the host must pass the address
// returned by cudaGetSymbolAddress to the kernels.
static __device__ __align__(256) double2 g_fft_mid[kMaxN];        // pass-1 output [N1][N2]
static __device__ __align__(256) double2 g_twiddle[kMaxN];        // exp(-2 pi i k / N)
// one entry per kept mode: 2 n_max + 1 <= n_fft - 1 < kMaxN
static __device__ __align__(256) double2 g_unit_phase[kMaxN];     // exp(i 0) per mode

struct DeviceScratch {
  bool ready = false;
  double2* mid = nullptr;
  double2* twiddle = nullptr;
  double2* unit_phase = nullptr;
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
DeviceScratch g_scratch[kMaxDevices];
swkb_status err(swkb_status s, const std::string& m) {
  swkb::set_last_error(m.c_str());
  return s;
}

__global__ void k_fill_twiddles(double2* tw, int N) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double s, c;
  sincospi(2.0 * (double)k / (double)N, &s, &c);
  tw[k] = make_double2(c, -s);
}

__global__ void k_fill_unit(double2* v, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[k] = make_double2(1.0, 0.0);
}

// Once per device, with that device current: resolve the device addresses of
// the scratch arrays and set the kernels' shared-memory limits.
swkb_status setup(int dev, DeviceScratch** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& d = g_scratch[dev];
  if (!d.ready) {
    cudaError_t e = cudaGetSymbolAddress((void**)&d.mid, g_fft_mid);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.twiddle, g_twiddle);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.unit_phase, g_unit_phase);
    if (e == cudaSuccess) e = swkb::prepare_fft_kernels<double>();
    if (e == cudaSuccess) {
      k_fill_unit<<<(kMaxN + 255) / 256, 256>>>(d.unit_phase, kMaxN);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
      return err(SWKB_ERR_CUDA, std::string("no-alloc set-up failed: ") + cudaGetErrorString(e));
    d.ready = true;
  }
  *out = &d;
  return SWKB_OK;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" swkb_status swkb_modes_noalloc(const double* u, int32_t n_fft, int32_t n_max,
                                          double* c, void* cuda_stream) {
  if (!u || !c) return err(SWKB_ERR_INVALID_ARG, "u and c must be device pointers");
  if (n_fft < 64 || n_fft > kMaxN || (n_fft & (n_fft - 1)))
    return err(SWKB_ERR_INVALID_ARG,
               "n_fft must be a power of two in [64, 65536] (the fixed scratch size)");
  if (n_max < 1 || n_max > n_fft / 2 - 1)
    return err(SWKB_ERR_INVALID_ARG, "n_max must be in [1, n_fft / 2 - 1]");
  if (!is_device_pointer(u) || !is_device_pointer(c))
    return err(SWKB_ERR_INVALID_ARG, "u and c must be device pointers");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(SWKB_ERR_CUDA, "no usable current device");
  DeviceScratch* d = nullptr;
  swkb_status st = setup(dev, &d);
  if (st != SWKB_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_fill_twiddles<<<(n_fft + 255) / 256, 256, 0, s>>>(d->twiddle, n_fft);
  e = cudaGetLastError();
  if (e != cudaSuccess) return err(SWKB_ERR_CUDA, cudaGetErrorString(e));
  swkb::FftArgs<double> f;
  f.u = reinterpret_cast<const double2*>(u);
  f.tw = d->twiddle;
  f.Y = d->mid;
  f.N = n_fft;
  f.N2 = n_fft < 2048 ? n_fft : 2048;   // N1 = n_fft / N2 <= 32
  f.mirror = 0;
  f.part = nullptr;   // the caller's field is read directly
  f.n_part = 0;
  f.sym = 0;
  f.W = nullptr;
  f.N1 = n_fft / f.N2;
  f.log2N2 = 0;
  while ((1 << f.log2N2) < f.N2) ++f.log2N2;
  f.n_max = n_max;
  f.inv_N = 1.0 / n_fft;
  f.ephi = d->unit_phase;
  f.c = reinterpret_cast<double2*>(c);
  f.cpol = nullptr;
  e = swkb::launch_fft<double>(f, s);
  if (e != cudaSuccess) return err(SWKB_ERR_CUDA, cudaGetErrorString(e));
  return SWKB_OK;
}
