// Patch-wise Fourier-continuation screens (Sec. 2.2, Eq. ifft_eq_phi_patches):
// the two kernels that replace the periodic DFT and resummation on a
// non-periodic interval.  The ray march and the bracket search are the
// periodic ones: a ray depends only on its mode angle and launch point, so
// one family per mode serves every patch.
//
//   k_fc_modes  one CTA per patch: the patch's samples, its FC-Gram
//               continuation to N_p = n_pat + C points, and the kept modes of
//               that sequence's DFT, w_n / N_p, rotated to the interval's
//               origin (exp(-2 pi i n s_p / N_p)) and carried over the screen
//               (exp(i k dx Pbar_n)): cf[p][n].  FP64 throughout (the
//               continuation operator's entries reach 3e3, so its
//               cancellations need FP64 even in mixed plans).
//   k_fc_resum  the interpolation fused with the modal sum, as the periodic
//               resummation, except that a ray's amplitude is complex: ray
//               (n, j) carries a_j (S^{p0}(z_j) cf[p0][n] + S^{p0+1}(z_j)
//               cf[p0+1][n]), p0 the first patch whose weight is non-zero at
//               z_j (at most two are), and the integer part of the phase is
//               2 pi (n m mod N_p) / N_p.
#include <cuda_runtime.h>

#include "swkb_device.cuh"
#include "swkb_fc_tables.h"

namespace swkb {

namespace {

constexpr int FC_MODES_THREADS = 256;
constexpr int FC_WARPS = 4;
constexpr int FC_CF = 16;   // X_w, X_{w+1}, phase b0..b3, Re a r0..r3, Im a i0..i3, 2 pad

template <typename T>
__host__ __device__ inline int fc_warp_bytes(int wcap) {
  return ((FC_CF + 4) * wcap * (int)sizeof(T) + 15) & ~15;
}

template <typename T>
__global__ void __launch_bounds__(FC_MODES_THREADS) k_fc_modes(const FcModesArgs<T> p) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* e = reinterpret_cast<double2*>(smem_raw);   // [N_p] the continued sequence
  double2* tw = e + p.Np;                              // [N_p] exp(-2 pi i k / N_p)
  const int pt = blockIdx.x;
  const long long s0 = (long long)pt * p.stride;
  for (int k = threadIdx.x; k < p.n_pat; k += blockDim.x) {
    const V v = p.u[s0 + k];
    e[k] = make_double2((double)v.x, (double)v.y);
  }
  for (int k = threadIdx.x; k < p.Np; k += blockDim.x) tw[k] = p.tw[k];
  __syncthreads();
  if (threadIdx.x < FC_C) {
    // value t past the right end: the right end's d samples through row t;
    // the same value counted backwards from the left end is C - t steps
    // before sample 0: the left end read backwards through row C - 1 - t
    const int t = threadIdx.x;
    double ar = 0.0, ai = 0.0;
    for (int i = 0; i < FC_D; ++i) {
      const double cr = p.cont[t * FC_D + i];
      const double cl = p.cont[(FC_C - 1 - t) * FC_D + i];
      const double2 fr = e[p.n_pat - FC_D + i];
      const double2 fl = e[FC_D - 1 - i];
      ar += cr * fr.x + cl * fl.x;
      ai += cr * fr.y + cl * fl.y;
    }
    e[p.n_pat + t] = make_double2(ar, ai);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned Np = (unsigned)p.Np;
  for (int i = warp; i < p.M; i += FC_MODES_THREADS / 32) {
    const int n = i - p.n_max;
    const unsigned nn = (unsigned)(((n % p.Np) + p.Np) % p.Np);
    const unsigned step = (unsigned)(((unsigned long long)nn * 32u) % Np);
    unsigned idx = (unsigned)(((unsigned long long)nn * (unsigned)lane) % Np);
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < p.Np; k += 32) {
      const double2 v = e[k], w = tw[idx];
      sr += v.x * w.x - v.y * w.y;
      si += v.x * w.y + v.y * w.x;
      idx += step;
      if (idx >= Np) idx -= Np;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_xor_sync(0xffffffffu, sr, o);
      si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const double2 rot = tw[(unsigned)(((unsigned long long)nn * (unsigned long long)s0) % Np)];
      const V ep = p.ephi[i];
      const double er = (double)ep.x, ei = (double)ep.y;
      // (sr + i si) rot exp(i phi) / N_p
      const double xr = sr * rot.x - si * rot.y, xi = sr * rot.y + si * rot.x;
      V c;
      c.x = (T)((xr * er - xi * ei) * p.inv_Np);
      c.y = (T)((xr * ei + xi * er) * p.inv_Np);
      p.cf[(long long)pt * p.M + i] = c;
    }
  }
}

__device__ __forceinline__ void store_row(float* r, float X1, float X2, float b0, float b1,
                                          float b2, float b3, float r0, float r1, float r2,
                                          float r3, float i0, float i1, float i2, float i3) {
  *reinterpret_cast<float4*>(r) = make_float4(X1, X2, b0, b1);
  *reinterpret_cast<float4*>(r + 4) = make_float4(b2, b3, r0, r1);
  *reinterpret_cast<float4*>(r + 8) = make_float4(r2, r3, i0, i1);
  *reinterpret_cast<float4*>(r + 12) = make_float4(i2, i3, 0.f, 0.f);
}
__device__ __forceinline__ void store_row(double* r, double X1, double X2, double b0, double b1,
                                          double b2, double b3, double r0, double r1, double r2,
                                          double r3, double i0, double i1, double i2,
                                          double i3) {
  *reinterpret_cast<double2*>(r) = make_double2(X1, X2);
  *reinterpret_cast<double2*>(r + 2) = make_double2(b0, b1);
  *reinterpret_cast<double2*>(r + 4) = make_double2(b2, b3);
  *reinterpret_cast<double2*>(r + 6) = make_double2(r0, r1);
  *reinterpret_cast<double2*>(r + 8) = make_double2(r2, r3);
  *reinterpret_cast<double2*>(r + 10) = make_double2(i0, i1);
  *reinterpret_cast<double2*>(r + 12) = make_double2(i2, i3);
}

template <typename T>
struct Row {
  T X1, X2, b0, b1, b2, b3, r0, r1, r2, r3, i0, i1, i2, i3;
};

template <typename T>
__device__ __forceinline__ Row<T> load_row(const T* r) {
  Row<T> o;
  if constexpr (sizeof(T) == 4) {
    const float4 a = *reinterpret_cast<const float4*>(r);
    const float4 b = *reinterpret_cast<const float4*>(r + 4);
    const float4 c = *reinterpret_cast<const float4*>(r + 8);
    const float2 d = *reinterpret_cast<const float2*>(r + 12);
    o = Row<T>{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y};
  } else {
    const double2 a = *reinterpret_cast<const double2*>(r);
    const double2 b = *reinterpret_cast<const double2*>(r + 2);
    const double2 c = *reinterpret_cast<const double2*>(r + 4);
    const double2 d = *reinterpret_cast<const double2*>(r + 6);
    const double2 f = *reinterpret_cast<const double2*>(r + 8);
    const double2 g = *reinterpret_cast<const double2*>(r + 10);
    const double2 h = *reinterpret_cast<const double2*>(r + 12);
    o = Row<T>{a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, f.x, f.y, g.x, g.y, h.x, h.y};
  }
  return o;
}

// One CTA: tile blk % n_tiles (TM = 32 PW points), mode group blk / n_tiles;
// its warps take the group's modes round-robin and the CTA adds the warps'
// sums in a fixed order.
template <typename T, int PW>
__global__ void __launch_bounds__(FC_WARPS * 32) k_fc_resum(const FcResumArgs<T> p) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = blockIdx.x % p.n_tiles, group = blockIdx.x / p.n_tiles;
  const int wcap = p.wcap, TM = p.TM, m0 = tile * TM;
  T* s_cf = reinterpret_cast<T*>(smem_raw + (long long)warp * fc_warp_bytes<T>(wcap));
  T* s_X = s_cf + FC_CF * wcap;
  T* s_ph = s_X + wcap;
  T* s_ar = s_ph + wcap;
  T* s_ai = s_ar + wcap;
  const int i0 = group * p.modes_per_group, i1 = min(p.M, i0 + p.modes_per_group);
  const unsigned Np = (unsigned)p.Np;
  const T invNp = T(1) / T(p.Np);
  const long long nrays = (long long)p.NRT * p.M;
  const long long njlo = (long long)(p.n_tiles + 1) * p.M;
  unsigned st = 0;
  T accr[PW], acci[PW];
#pragma unroll
  for (int q = 0; q < PW; ++q) { accr[q] = T(0); acci[q] = T(0); }

  for (int i = i0 + warp; i < i1; i += FC_WARPS) {
    const int jl = p.jlo[bchk((long long)tile * p.M + i, njlo, st)];
    const int jh = p.jlo[bchk((long long)(tile + 1) * p.M + i, njlo, st)];
    // a table left inconsistent by a failed screen (flagged by the bracket
    // kernel) must not send the reads out of [0, NRT)
    if (jl < 1 || jh < jl || jh > p.NRT - 3) continue;
    const int W = jh - jl + 4;
    if (W > wcap) { st |= ST_CAUSTIC; continue; }
    const int jb = jl - 1;
    __syncwarp();
    for (int w = lane; w < W; w += 32) {
      const int j = jb + w;
      const long long o = bchk((long long)j * p.M + i, nrays, st);
      s_X[w] = T((j - p.G) * p.R - m0) + ld<LD_NC>(p.d + o);
      s_ph[w] = ld<LD_NC>(p.ph + o);
      const T a = ld<LD_NC>(p.a + o);
      const int p0 = p.win_p[j];
      const V s = p.win_s[j];
      const V c0 = p.cf[bchk((long long)p0 * p.M + i, (long long)p.P * p.M, st)];
      T cr = s.x * c0.x, ci = s.x * c0.y;
      if (p0 + 1 < p.P) {
        const V c1 = p.cf[(long long)(p0 + 1) * p.M + i];
        cr += s.y * c1.x;
        ci += s.y * c1.y;
      }
      s_ar[w] = a * cr;
      s_ai[w] = a * ci;
    }
    __syncwarp();
    for (int w = 1 + lane; w <= W - 3; w += 32) {
      const T X0 = s_X[w - 1], X1 = s_X[w], X2 = s_X[w + 1], X3 = s_X[w + 2];
      const T h21 = X2 - X1, h10 = X1 - X0;
      const T r21 = T(1) / h21, r10 = T(1) / h10, r32 = T(1) / (X3 - X2);
      const T r20 = T(1) / (X2 - X0), r31 = T(1) / (X3 - X1), r30 = T(1) / (X3 - X0);
      T b0, b1, b2, b3, c0, c1, c2, c3, d0, d1, d2, d3;
      cubic_through(s_ph[w - 1], s_ph[w], s_ph[w + 1], s_ph[w + 2], r21, r10, r32, r20, r31, r30,
                    h21, h10, b0, b1, b2, b3);
      cubic_through(s_ar[w - 1], s_ar[w], s_ar[w + 1], s_ar[w + 2], r21, r10, r32, r20, r31, r30,
                    h21, h10, c0, c1, c2, c3);
      cubic_through(s_ai[w - 1], s_ai[w], s_ai[w + 1], s_ai[w + 2], r21, r10, r32, r20, r31, r30,
                    h21, h10, d0, d1, d2, d3);
      if constexpr (sizeof(T) == 4) b0 = minus_rint(b0);   // whole turns do not matter
      store_row(s_cf + FC_CF * w, X1, X2, b0, b1, b2, b3, c0, c1, c2, c3, d0, d1, d2, d3);
    }
    __syncwarp();
    // lane l sums the PW consecutive points l PW .. l PW + PW - 1 of the tile
    const T xf = s_X[1];
    const T inv_sp = T(W - 3) / (s_X[W - 2] - xf);
    const int x0 = lane * PW;
    const T xv0 = T(x0);
    int w = 1 + ifloor_small(xv0 * inv_sp - xf * inv_sp);
    w = min(max(w, 1), W - 3);
    while (w > 1 && s_X[w] > xv0) --w;
    while (w < W - 3 && s_X[w + 1] <= xv0) ++w;
    Row<T> r = load_row<T>(s_cf + FC_CF * w);
    const int n = i - p.n_max;
    const unsigned nn = (unsigned)(((n % p.Np) + p.Np) % p.Np);
    unsigned nm = (unsigned)(((unsigned long long)nn * (unsigned long long)(m0 + x0)) % Np);
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const T xv = xv0 + T(q);
      while (w < W - 3 && r.X2 <= xv) {
        ++w;
        r = load_row<T>(s_cf + FC_CF * w);
      }
      const T tau = xv - r.X1;
      const T phv = ((r.b3 * tau + r.b2) * tau + r.b1) * tau + r.b0;
      const T ar = ((r.r3 * tau + r.r2) * tau + r.r1) * tau + r.r0;
      const T ai = ((r.i3 * tau + r.i2) * tau + r.i1) * tau + r.i0;
      const T t = minus_rint(T(nm) * invNp + phv);
      T sn, cs;
      sincos_turns(t, &sn, &cs);
      accr[q] += ar * cs - ai * sn;
      acci[q] += ar * sn + ai * cs;
      nm += nn;
      if (nm >= Np) nm -= Np;
    }
  }
  __syncthreads();
  V* red = reinterpret_cast<V*>(smem_raw);
  const int TMP = 32 * (PW + 1);
#pragma unroll
  for (int q = 0; q < PW; ++q) {
    V v;
    v.x = accr[q];
    v.y = acci[q];
    red[warp * TMP + lane * (PW + 1) + q] = v;
  }
  __syncthreads();
  V* out = p.part + bchk((long long)group * p.N + m0, (long long)p.n_groups * p.N - (TM - 1), st);
  if (st) atomicOr(p.status, st);
  for (int x = threadIdx.x; x < TM; x += FC_WARPS * 32) {
    const int xs = (x / PW) * (PW + 1) + x % PW;
    V sum = red[xs];
#pragma unroll
    for (int k = 1; k < FC_WARPS; ++k) {
      const V v = red[k * TMP + xs];
      sum.x += v.x;
      sum.y += v.y;
    }
    out[x] = sum;
  }
}

template <typename T, int PW>
cudaError_t resum_pw(const FcResumArgs<T>& a, cudaStream_t s) {
  const size_t smem = fc_resum_smem_bytes<T>(a.wcap, a.TM);
  k_fc_resum<T, PW><<<a.n_tiles * a.n_groups, FC_WARPS * 32, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
size_t fc_resum_smem_bytes(int wcap, int tile_points) {
  const size_t rows = (size_t)FC_WARPS * fc_warp_bytes<T>(wcap);
  const int PW = tile_points / 32;
  const size_t red = (size_t)FC_WARPS * 32 * (PW + 1) * 2 * sizeof(T);
  return rows > red ? rows : red;
}

template <typename T>
size_t fc_modes_smem_bytes(int Np) {
  return 2 * (size_t)Np * sizeof(double2);
}

template <typename T>
cudaError_t prepare_fc_kernels(int resum_smem, int modes_smem) {
  cudaError_t e = cudaFuncSetAttribute(k_fc_modes<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       modes_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fc_resum<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           resum_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_fc_resum<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           resum_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_fc_resum<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              resum_smem);
}

template <typename T>
cudaError_t launch_fc_modes(const FcModesArgs<T>& a, cudaStream_t s) {
  k_fc_modes<T><<<a.P, FC_MODES_THREADS, fc_modes_smem_bytes<T>(a.Np), s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fc_resum(const FcResumArgs<T>& a, cudaStream_t s) {
  switch (a.TM / 32) {
    case 2: return resum_pw<T, 2>(a, s);
    case 4: return resum_pw<T, 4>(a, s);
    case 8: return resum_pw<T, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

const double* fc_continuation_host() { return &kFcContinuation[0][0]; }

template size_t fc_resum_smem_bytes<float>(int, int);
template size_t fc_resum_smem_bytes<double>(int, int);
template size_t fc_modes_smem_bytes<float>(int);
template size_t fc_modes_smem_bytes<double>(int);
template cudaError_t prepare_fc_kernels<float>(int, int);
template cudaError_t prepare_fc_kernels<double>(int, int);
template cudaError_t launch_fc_modes<float>(const FcModesArgs<float>&, cudaStream_t);
template cudaError_t launch_fc_modes<double>(const FcModesArgs<double>&, cudaStream_t);
template cudaError_t launch_fc_resum<float>(const FcResumArgs<float>&, cudaStream_t);
template cudaError_t launch_fc_resum<double>(const FcResumArgs<double>&, cudaStream_t);

}  // namespace swkb
