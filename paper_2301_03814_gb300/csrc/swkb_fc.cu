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
//               (exp(i k dx Pbar_n)): cf[p][n].  The continuation runs in
//               FP64 in every plan (the operator's entries reach 3e3, so its
//               cancellations need FP64); the DFT sums in the plan's type.
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
constexpr int FC_MODES_PER_CTA = 64;   // 8 warps x 8 modes
constexpr int FC_WARPS = 4;
constexpr int FC_PF = 2;    // rounds of 32 rays prefetched one mode ahead
// Row of interval w: X_w, X_{w+1}, phase b0..b3, Re a r0..r3, Im a i0..i3.
// 14 values accessed as 7 pairs: at a 56-byte (FP32) row stride the 16
// lanes of a half-warp touch 32 distinct banks.
constexpr int FC_CF = 14;

// x mod Np for x < 2^32 with magic = floor(2^32 / Np): the quotient
// estimate is floor(x / Np) or one less, so one correction finishes it.
__device__ __forceinline__ unsigned mod_np(unsigned x, unsigned Np, unsigned magic) {
  unsigned r = x - __umulhi(x, magic) * Np;
  return r >= Np ? r - Np : r;
}

template <typename T>
__host__ __device__ inline int fc_warp_bytes(int wcap) {
  return ((FC_CF + 4) * wcap * (int)sizeof(T) + 15) & ~15;
}

// CTA (patch blockIdx.x, mode block blockIdx.y): the continuation in FP64,
// then the DFT of the FC_MODES_PER_CTA modes of the block in T (a mixed plan
// sums in FP32: exact twiddle indices, FP32 twiddles and samples).
template <typename T>
__global__ void __launch_bounds__(FC_MODES_THREADS) k_fc_modes(const FcModesArgs<T> p) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* e = reinterpret_cast<V*>(smem_raw);    // [N_p] the continued sequence
  V* tw = e + p.Np;                         // [N_p] exp(-2 pi i k / N_p)
  __shared__ double2 ends[2 * FC_D];        // the d samples at each end, FP64
  const int pt = blockIdx.x;
  const long long s0 = (long long)pt * p.stride;
  for (int k = threadIdx.x; k < p.n_pat; k += blockDim.x) {
    const V v = p.u[s0 + k];
    e[k] = v;
    if (k < FC_D) ends[FC_D + k] = make_double2((double)v.x, (double)v.y);
    if (k >= p.n_pat - FC_D) ends[k - (p.n_pat - FC_D)] = make_double2((double)v.x, (double)v.y);
  }
  for (int k = threadIdx.x; k < p.Np; k += blockDim.x) {
    const double2 w = p.tw[k];
    V v;
    v.x = (T)w.x;
    v.y = (T)w.y;
    tw[k] = v;
  }
  __syncthreads();
  if (threadIdx.x < FC_C) {
    // value t past the right end: the right end's d samples (ends[0 .. d-1])
    // through row t; the same value counted backwards from the left end is
    // C - t steps before sample 0: the left end read backwards (sample
    // d - 1 - i = ends[2 d - 1 - i]) through row C - 1 - t
    const int t = threadIdx.x;
    double ar = 0.0, ai = 0.0;
    for (int i = 0; i < FC_D; ++i) {
      const double cr = p.cont[t * FC_D + i];
      const double cl = p.cont[(FC_C - 1 - t) * FC_D + i];
      const double2 fr = ends[i];
      const double2 fl = ends[2 * FC_D - 1 - i];
      ar += cr * fr.x + cl * fl.x;
      ai += cr * fr.y + cl * fl.y;
    }
    V v;
    v.x = (T)ar;
    v.y = (T)ai;
    e[p.n_pat + t] = v;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned Np = (unsigned)p.Np;
  const int i_end = min(p.M, (int)(blockIdx.y + 1) * FC_MODES_PER_CTA);
  for (int i = blockIdx.y * FC_MODES_PER_CTA + warp; i < i_end; i += FC_MODES_THREADS / 32) {
    const int n = i - p.n_max;   // |n| < Np / 2
    const unsigned nn = (unsigned)(n < 0 ? n + p.Np : n);
    const unsigned step = mod_np(nn * 32u, Np, p.np_magic);
    unsigned idx = mod_np(nn * (unsigned)lane, Np, p.np_magic);
    T sr = T(0), si = T(0);
    for (int k = lane; k < p.Np; k += 32) {
      const V v = e[k], w = tw[idx];
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
      // (sr + i si) rot exp(i phi) / N_p in the plan's type; nn s0 < 2^11 2^20
      const V rot = tw[mod_np(nn * (unsigned)s0, Np, p.np_magic)];
      const V ep = p.ephi[i];
      const T xr = sr * rot.x - si * rot.y, xi = sr * rot.y + si * rot.x;
      const T inv = (T)p.inv_Np;
      V c;
      c.x = (xr * ep.x - xi * ep.y) * inv;
      c.y = (xr * ep.y + xi * ep.x) * inv;
      p.cf[(long long)pt * p.M + i] = c;
    }
  }
}

template <typename T>
__device__ __forceinline__ void store_row(T* r, T X1, T X2, T b0, T b1, T b2, T b3, T r0, T r1,
                                          T r2, T r3, T i0, T i1, T i2, T i3) {
  using V = typename C2<T>::type;
  V* q = reinterpret_cast<V*>(r);
  q[0] = V{X1, X2};
  q[1] = V{b0, b1};
  q[2] = V{b2, b3};
  q[3] = V{r0, r1};
  q[4] = V{r2, r3};
  q[5] = V{i0, i1};
  q[6] = V{i2, i3};
}

template <typename T>
struct Row {
  T X1, X2, b0, b1, b2, b3, r0, r1, r2, r3, i0, i1, i2, i3;
};

template <typename T>
__device__ __forceinline__ Row<T> load_row(const T* r) {
  using V = typename C2<T>::type;
  const V* q = reinterpret_cast<const V*>(r);
  const V a = q[0], b = q[1], c = q[2], d = q[3], e = q[4], f = q[5], g = q[6];
  return Row<T>{a.x, a.y, b.x, b.y, c.x, c.y, d.x, d.y, e.x, e.y, f.x, f.y, g.x, g.y};
}

// One CTA: tile blk % n_tiles (TM = 32 PW points), mode group blk / n_tiles;
// its warps take the group's modes round-robin and the CTA adds the warps'
// sums in a fixed order.
// FP32: at most 80 registers per thread (measured faster than the
// unbounded 93: 0.31 against 0.47 ms per sum on a 131072-point open lens)
template <typename T, int PW>
__global__ void __launch_bounds__(FC_WARPS * 32, sizeof(T) == 4 ? 6 : 1)
    k_fc_resum(const FcResumArgs<T> p) {
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

  // ray j of mode i: landing offset, phase and the complex amplitude
  // a_j (S^{p0}(z_j) cf[p0][i] + S^{p0+1}(z_j) cf[p0+1][i])
  auto fetch = [&](int i, int j, T& d, T& ph, T& ar, T& ai) {
    // NRT M < 2^32 (at most 2^20 + 2 G rays of 2047 modes)
    const unsigned o = (unsigned)bchk((long long)((unsigned)j * (unsigned)p.M + (unsigned)i),
                                      nrays, st);
    d = ld<LD_NC>(p.d + o);
    ph = ld<LD_NC>(p.ph + o);
    const T a = ld<LD_NC>(p.a + o);
    const int p0 = p.win_p[j];
    const V sw = p.win_s[j];
    const V c0 = p.cf[bchk((long long)p0 * p.M + i, (long long)p.P * p.M, st)];
    T cr = sw.x * c0.x, ci = sw.x * c0.y;
    if (p0 + 1 < p.P) {
      const V c1 = p.cf[(long long)(p0 + 1) * p.M + i];
      cr += sw.y * c1.x;
      ci += sw.y * c1.y;
    }
    ar = a * cr;
    ai = a * ci;
  };
  auto head = [&](int i, int& jl, int& jh) {
    jl = -1;
    jh = -1;
    if (i >= i1) return;
    jl = p.jlo[bchk((long long)tile * p.M + i, njlo, st)];
    jh = p.jlo[bchk((long long)(tile + 1) * p.M + i, njlo, st)];
  };
  // a table left inconsistent by a failed screen (flagged by the bracket
  // kernel) must not send the reads out of [0, NRT); a window beyond the
  // tile's capacity means rays compressed beyond it (flagged here)
  auto head_ok = [&](int i, int jl, int jh) {
    if (i >= i1 || jl < 1 || jh < jl || jh > p.NRT - 3) return false;
    if (jh - jl + 4 > wcap) {
      st |= ST_CAUSTIC;
      return false;
    }
    return true;
  };
  // the next mode's first FC_PF rounds of 32 rays are loaded into registers
  // while the current mode is summed
  T pd[FC_PF], pph[FC_PF], par[FC_PF], pai[FC_PF];
  auto prefetch = [&](int i, int jl, int jh) {
    const int W = jh - jl + 4;
#pragma unroll
    for (int r = 0; r < FC_PF; ++r) {
      const int w = lane + 32 * r;
      if (w < W) fetch(i, jl - 1 + w, pd[r], pph[r], par[r], pai[r]);
    }
  };

  int i = i0 + warp;
  int jl_c, jh_c, jl_n, jh_n;
  head(i, jl_c, jh_c);
  head(i + FC_WARPS, jl_n, jh_n);
  bool ok_c = head_ok(i, jl_c, jh_c);
  if (ok_c) prefetch(i, jl_c, jh_c);
  for (; i < i1; i += FC_WARPS) {
    const bool ok = ok_c;
    const int jl = jl_c, jh = jh_c;
    const int W = jh - jl + 4;
    const int jb = jl - 1;
    __syncwarp();
    if (ok) {
#pragma unroll
      for (int r = 0; r < FC_PF; ++r) {
        const int w = lane + 32 * r;
        if (w < W) {
          s_X[w] = T((jb + w - p.G) * p.R - m0) + pd[r];
          s_ph[w] = pph[r];
          s_ar[w] = par[r];
          s_ai[w] = pai[r];
        }
      }
      for (int w = lane + 32 * FC_PF; w < W; w += 32) {
        T d, ph, ar, ai;
        fetch(i, jb + w, d, ph, ar, ai);
        s_X[w] = T((jb + w - p.G) * p.R - m0) + d;
        s_ph[w] = ph;
        s_ar[w] = ar;
        s_ai[w] = ai;
      }
    }
    jl_c = jl_n;
    jh_c = jh_n;
    ok_c = head_ok(i + FC_WARPS, jl_c, jh_c);
    if (ok_c) prefetch(i + FC_WARPS, jl_c, jh_c);
    head(i + 2 * FC_WARPS, jl_n, jh_n);
    if (!ok) continue;
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
    const int n = i - p.n_max;   // |n| < Np / 2
    const unsigned nn = (unsigned)(n < 0 ? n + p.Np : n);
    if constexpr (sizeof(T) == 4) {
      // the exact integer phase n m / Np mod 1 of the run's middle point,
      // moved into [-1/2, 1/2), and n / Np (|n / Np| < 1/2) per point from it:
      // the argument of the sine stays within about two turns
      const unsigned nmc = mod_np(nn * (unsigned)(m0 + x0 + PW / 2), Np, p.np_magic);
      T bc = T(nmc) * invNp;
      bc = bc >= T(0.5) ? bc - T(1) : bc;
      const T nNp = T(n) * invNp;
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
        const T t = fmaf(T(q - PW / 2), nNp, bc) + phv;
        T sn, cs;
        sincos_turns(t, &sn, &cs);
        accr[q] += ar * cs - ai * sn;
        acci[q] += ar * sn + ai * cs;
      }
    } else {
      // nn (m0 + x0) < 2^11 2^20: no overflow
      unsigned nm = mod_np(nn * (unsigned)(m0 + x0), Np, p.np_magic);
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
  return 2 * (size_t)Np * sizeof(typename C2<T>::type);
}

template <typename T>
cudaError_t prepare_fc_kernels(int resum_smem, int modes_smem) {
  // The limit is a per-device property of the kernel shared by every plan in
  // the process: raise it to the device's opt-in maximum (never lower it, or a
  // plan with a shorter period or smaller tiles would break another plan's
  // launches).
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (resum_smem > optin || modes_smem + (int)(2 * FC_D * sizeof(double2)) > optin)
    return cudaErrorInvalidValue;
  const void* fs[] = {(const void*)k_fc_modes<T>, (const void*)k_fc_resum<T, 2>,
                      (const void*)k_fc_resum<T, 4>, (const void*)k_fc_resum<T, 8>};
  for (const void* f : fs) {
    // the dynamic limit plus the kernel's static shared memory must stay
    // within the opt-in maximum
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// out[p][n] = cf[p][n] f[n]: the patches' coefficients carried to a plane
// inside the screen (f: exp(i k (j / P - 1) dx Pbar_n)).
template <typename T>
__global__ void k_fc_cscale(const typename C2<T>::type* __restrict__ cf,
                            const typename C2<T>::type* __restrict__ f,
                            typename C2<T>::type* __restrict__ out, int PM, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= PM) return;
  const typename C2<T>::type a = cf[k], b = f[k % M];
  typename C2<T>::type c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  out[k] = c;
}

template <typename T>
cudaError_t launch_fc_cscale(const typename C2<T>::type* cf, const typename C2<T>::type* f,
                             typename C2<T>::type* out, int P, int M, cudaStream_t s) {
  const int PM = P * M;
  k_fc_cscale<T><<<(PM + 255) / 256, 256, 0, s>>>(cf, f, out, PM, M);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fc_modes(const FcModesArgs<T>& a, cudaStream_t s) {
  const dim3 grid(a.P, (a.M + FC_MODES_PER_CTA - 1) / FC_MODES_PER_CTA);
  k_fc_modes<T><<<grid, FC_MODES_THREADS, fc_modes_smem_bytes<T>(a.Np), s>>>(a);
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
template cudaError_t launch_fc_cscale<float>(const float2*, const float2*, float2*, int, int,
                                             cudaStream_t);
template cudaError_t launch_fc_cscale<double>(const double2*, const double2*, double2*, int, int,
                                              cudaStream_t);
template cudaError_t launch_fc_resum<double>(const FcResumArgs<double>&, cudaStream_t);

}  // namespace swkb
