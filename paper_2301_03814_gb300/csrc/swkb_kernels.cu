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

#include <math.h>
#include <stdint.h>

#include "swkb_internal.h"

namespace swkb {

// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------
__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

template <typename T>
__device__ __forceinline__ void load6(const T* p, T& a0, T& a1, T& a2, T& a3, T& a4, T& a5);

template <>
__device__ __forceinline__ void load6<float>(const float* p, float& a0, float& a1, float& a2,
                                             float& a3, float& a4, float& a5) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  const float2 w = __ldg(reinterpret_cast<const float2*>(p + 4));
  a0 = v.x; a1 = v.y; a2 = v.z; a3 = v.w; a4 = w.x; a5 = w.y;
}

template <>
__device__ __forceinline__ void load6<double>(const double* p, double& a0, double& a1, double& a2,
                                              double& a3, double& a4, double& a5) {
  const double2 u = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v = __ldg(reinterpret_cast<const double2*>(p + 2));
  const double2 w = __ldg(reinterpret_cast<const double2*>(p + 4));
  a0 = u.x; a1 = u.y; a2 = v.x; a3 = v.y; a4 = w.x; a5 = w.y;
}

// ----------------------------------------------------------------------------
// medium: quintic in z per interval, linear in x between two columns
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void col_eval(const Medium<T>& m, int c, T zz, T& e, T& ez, T& ezz,
                                         unsigned& st) {
  const T u = (zz - m.z0) * m.inv_h;
  int i;
  T t;
  if (!(u >= T(0))) {                       // below the table (or NaN)
    st |= ST_RANGE; i = 0; t = T(0);
  } else {
    const T fi = floor(u);
    if (fi >= T(m.n_int)) {
      if (!(fi == T(m.n_int) && u == fi)) st |= ST_RANGE;
      i = m.n_int - 1; t = T(1);
    } else {
      i = (int)fi; t = u - fi;
    }
  }
  T a0, a1, a2, a3, a4, a5;
  load6<T>(m.coef + (long long)c * m.col_stride + (long long)i * 8, a0, a1, a2, a3, a4, a5);
  e = a0 + t * (a1 + t * (a2 + t * (a3 + t * (a4 + t * a5))));
  ez = (a1 + t * (T(2) * a2 + t * (T(3) * a3 + t * (T(4) * a4 + t * (T(5) * a5))))) * m.inv_h;
  ezz = (T(2) * a2 + t * (T(6) * a3 + t * (T(12) * a4 + t * (T(20) * a5)))) * m.inv_h2;
}

// eps - eps_ref, eps_z, eps_zz at RK4 stage l and height z.
template <typename T>
__device__ __forceinline__ void medium_eval(const MarchArgs<T>& p, int l, T z, T& e, T& ez,
                                            T& ezz, unsigned& st) {
  T zz = z, sg = T(1);
  if (p.med.mirrored) {
    const T d = z - p.med.z_mirror;
    sg = d < T(0) ? T(-1) : T(1);
    zz = p.med.z_mirror + fabs(d);
  }
  const int c = __ldg(p.st.c + l);
  const T th = __ldg(p.st.th + l);
  if (th == T(0)) {
    col_eval(p.med, c, zz, e, ez, ezz, st);
  } else if (th == T(1)) {
    col_eval(p.med, c + 1, zz, e, ez, ezz, st);
  } else {
    T e0, ez0, ezz0, e1, ez1, ezz1;
    col_eval(p.med, c, zz, e0, ez0, ezz0, st);
    col_eval(p.med, c + 1, zz, e1, ez1, ezz1, st);
    e = (T(1) - th) * e0 + th * e1;
    ez = (T(1) - th) * ez0 + th * ez1;
    ezz = (T(1) - th) * ezz0 + th * ezz1;
  }
  ez *= sg;
}

// ----------------------------------------------------------------------------
// (b) ray march
// ----------------------------------------------------------------------------
template <typename T>
struct Ray {
  T dz, dQ, rh, Zs, Qs;
};

// x-form right-hand side (Eqs. charsys / charsys_s divided by x_t = 2P):
//   z' = Q/P, Q' = eps_z/(2P), r' = (eps - kappa Q)/P,
//   P_s = (eps_z Z_s - 2 Q Q_s)/(2P), Z_s' = (Q_s - Q P_s/P)/P,
//   Q_s' = (eps_zz Z_s - eps_z P_s/P)/(2P)
// in deviation form: with e = eps - eps_ref and D = e - dQ (2 kappa + dQ),
// P^2 = P_bar^2 + D and r' - P_bar = (e - kappa dQ - P_bar D/(P_bar + P))/P.
template <typename T>
__device__ __forceinline__ Ray<T> rhs(const MarchArgs<T>& p, int l, T s, T kap, T pb, T pb2,
                                      const Ray<T>& y, unsigned& st) {
  T e, ez, ezz;
  medium_eval(p, l, s + y.dz, e, ez, ezz, st);
  const T Q = kap + y.dQ;
  const T D = e - y.dQ * (T(2) * kap + y.dQ);
  T P2 = pb2 + D;
  if (!(P2 > T(0))) { st |= ST_TURNING; P2 = pb2; }
  if (!(y.Zs > T(0))) st |= ST_CAUSTIC;
  const T P = sqrt(P2);
  const T iP = T(1) / P;
  Ray<T> d;
  d.dz = Q * iP;
  d.dQ = T(0.5) * ez * iP;
  d.rh = (e - kap * y.dQ - pb * D / (pb + P)) * iP;
  const T PsiP = (ez * y.Zs - T(2) * Q * y.Qs) * (T(0.5) * iP) * iP;   // P_s / P
  d.Zs = (y.Qs - Q * PsiP) * iP;
  d.Qs = T(0.5) * (ezz * y.Zs - ez * PsiP) * iP;
  return d;
}

template <typename T>
__device__ __forceinline__ Ray<T> axpy(const Ray<T>& y, T a, const Ray<T>& k) {
  return Ray<T>{y.dz + a * k.dz, y.dQ + a * k.dQ, y.rh + a * k.rh, y.Zs + a * k.Zs,
                y.Qs + a * k.Qs};
}

// Block (32, 8): lanes are 32 consecutive modes at one launch height, so a
// warp's table reads stay within a few z-intervals; warps are 8 rays.
template <typename T>
__global__ void __launch_bounds__(256) k_march(const MarchArgs<T> p) {
  const int i = blockIdx.x * 32 + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= p.M || j >= p.NRT) return;
  unsigned st = 0;
  const T kap = p.kappa[i], pb = p.pbar[i], pb2 = p.pbar2[i];
  const T s = p.z_lo + T((j - p.G) * p.R) * p.dz;
  T e, ez, ezz;
  medium_eval(p, 0, s, e, ez, ezz, st);
  T P0sq = pb2 + e;
  if (!(P0sq > T(0))) { st |= ST_TURNING; P0sq = pb2; }
  const T P0 = sqrt(P0sq);
  Ray<T> y{T(0), T(0), T(0), T(1), T(0)};
  const T h = p.h, hh = T(0.5) * p.h, h6 = p.h / T(6);
  for (int n = 0; n < p.Nt; ++n) {
    const Ray<T> k1 = rhs(p, 2 * n, s, kap, pb, pb2, y, st);
    const Ray<T> k2 = rhs(p, 2 * n + 1, s, kap, pb, pb2, axpy(y, hh, k1), st);
    const Ray<T> k3 = rhs(p, 2 * n + 1, s, kap, pb, pb2, axpy(y, hh, k2), st);
    const Ray<T> k4 = rhs(p, 2 * n + 2, s, kap, pb, pb2, axpy(y, h, k3), st);
    y.dz += h6 * (k1.dz + T(2) * k2.dz + T(2) * k3.dz + k4.dz);
    y.dQ += h6 * (k1.dQ + T(2) * k2.dQ + T(2) * k3.dQ + k4.dQ);
    y.rh += h6 * (k1.rh + T(2) * k2.rh + T(2) * k3.rh + k4.rh);
    y.Zs += h6 * (k1.Zs + T(2) * k2.Zs + T(2) * k3.Zs + k4.Zs);
    y.Qs += h6 * (k1.Qs + T(2) * k2.Qs + T(2) * k3.Qs + k4.Qs);
  }
  if (!(y.Zs > T(0))) st |= ST_CAUSTIC;
  medium_eval(p, 2 * p.Nt, s + y.dz, e, ez, ezz, st);
  T P1sq = pb2 + e - y.dQ * (T(2) * kap + y.dQ);
  if (!(P1sq > T(0))) { st |= ST_TURNING; P1sq = pb2; }
  const T Zs = y.Zs > T(0) ? y.Zs : T(1);
  const long long o = (long long)j * p.M + i;
  p.out_d[o] = y.dz * p.inv_dz;
  p.out_ph[o] = y.rh * p.k_over_2pi;
  p.out_a[o] = sqrt(P0 / (sqrt(P1sq) * Zs));
  if (st) atomicOr(p.status, st);
}

// ----------------------------------------------------------------------------
// landing checks and tile brackets
// ----------------------------------------------------------------------------
// Landing of ray j in grid units: g_j = (j - G) R + d_j.  Tile t starts at
// grid point t TM; jlo[t][i] = the j with g_j <= t TM < g_{j+1}.
template <typename T>
__global__ void k_bracket(const BracketArgs<T> p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (i >= p.M || j >= p.NRT - 1) return;
  const T d0 = p.d[(long long)j * p.M + i];
  const T d1 = p.d[(long long)(j + 1) * p.M + i];
  const long long b0 = (long long)(j - p.G) * p.R;
  const long long b1 = b0 + p.R;
  unsigned st = 0;
  if (!(T(p.R) + d1 - d0 > T(0))) st |= ST_CAUSTIC;                  // g_{j+1} > g_j
  if (j == 1 && !(d0 <= T(-b0))) st |= ST_COVER;                      // g_1 <= 0
  if (j + 1 == p.NRT - 2 && !(d1 > T((long long)p.N - b1))) st |= ST_COVER;  // g_{NRT-2} > N
  if (st) {
    atomicOr(p.status, st);
    return;
  }
  const long long TM = p.TM;
  long long t0 = (long long)ceil(((double)b0 + (double)d0) / (double)TM);
  long long t1 = (long long)ceil(((double)b1 + (double)d1) / (double)TM) - 1;
  t0 = t0 < -1 ? -1 : (t0 > p.n_tiles + 1 ? p.n_tiles + 1 : t0);
  t1 = t1 < -1 ? -1 : (t1 > p.n_tiles + 1 ? p.n_tiles + 1 : t1);
  // exact fix-ups: t0 = min t with t TM >= g_j, t1 = max t with t TM < g_{j+1}
  for (int k = 0; k < 4 && d0 <= T((t0 - 1) * TM - b0); ++k) --t0;
  for (int k = 0; k < 4 && !(d0 <= T(t0 * TM - b0)); ++k) ++t0;
  for (int k = 0; k < 4 && !(T(t1 * TM - b1) < d1); ++k) --t1;
  for (int k = 0; k < 4 && T((t1 + 1) * TM - b1) < d1; ++k) ++t1;
  if (t0 < 0) t0 = 0;
  if (t1 > p.n_tiles) t1 = p.n_tiles;
  for (long long t = t0; t <= t1; ++t) p.jlo[t * p.M + i] = j;
}

// ----------------------------------------------------------------------------
// (c) + (d) interpolation fused with the modal sum
// ----------------------------------------------------------------------------
// One warp owns TM = 32 PW consecutive grid points (PW per lane) of one tile
// and sums the modes of one mode group into registers.  For every mode the
// rays landing on the tile (brackets jlo[t] .. jlo[t+1], stencil -1 / +2) are
// staged in shared memory (a global-memory view is used if they do not fit);
// each lane walks its bracket, builds the Newton form of the 4-point Lagrange
// polynomial through the stencil (nodes x_{j-1}, x_j, x_{j+1}, x_{j+2}), and
// evaluates phase and amplitude at its points.  The phase of term (n, m) is
// exact in its integer part: k kappa_n (z_m - z_lo) = 2 pi (n m mod N) / N.
template <typename T, int PW>
__global__ void __launch_bounds__(128) k_resum(const ResumArgs<T> p) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int item = blockIdx.x * (blockDim.x >> 5) + warp;
  if (item >= p.n_tiles * p.n_groups) return;
  const int tile = item % p.n_tiles;
  const int group = item / p.n_tiles;
  T* s_d = reinterpret_cast<T*>(smem_raw) + (long long)warp * 3 * p.wcap;
  T* s_ph = s_d + p.wcap;
  T* s_a = s_ph + p.wcap;
  const int m0 = tile * p.TM;
  const int i0 = group * p.modes_per_group;
  const int i1 = min(p.M, i0 + p.modes_per_group);
  const T invN = T(1) / T(p.N);
  const unsigned mask = (unsigned)p.N - 1u;

  T accr[PW], acci[PW];
#pragma unroll
  for (int q = 0; q < PW; ++q) { accr[q] = T(0); acci[q] = T(0); }

  for (int i = i0; i < i1; ++i) {
    const int jl = __ldg(p.jlo + (long long)tile * p.M + i);
    const int jh = __ldg(p.jlo + (long long)(tile + 1) * p.M + i);
    // A bracket table left inconsistent by a failed screen (already flagged
    // by k_bracket) must not send the reads out of [0, NRT).
    if (jl < 1 || jh < jl || jh > p.NRT - 3) continue;
    const int jb = jl - 1;
    const int W = jh - jl + 4;
    const T* gd;
    const T* gph;
    const T* ga;
    long long stride;
    __syncwarp();
    if (W <= p.wcap) {
      for (int w = lane; w < W; w += 32) {
        const long long o = (long long)(jb + w) * p.M + i;
        s_d[w] = __ldg(p.d + o);
        s_ph[w] = __ldg(p.ph + o);
        s_a[w] = __ldg(p.a + o);
      }
      __syncwarp();
      gd = s_d; gph = s_ph; ga = s_a; stride = 1;
    } else {
      const long long o = (long long)jb * p.M + i;
      gd = p.d + o; gph = p.ph + o; ga = p.a + o; stride = p.M;
    }
    const int base = (jb - p.G) * p.R - m0;   // node w sits at base + w R + d_w
    const T x0 = T(lane * PW);
    int lo = 1, hi = W - 2;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (T(base + mid * p.R) + gd[mid * stride] <= x0) lo = mid; else hi = mid;
    }
    int wb = lo;
    int cur = -1;
    T X1 = 0, h21 = 0, h10 = 0;
    T cp0 = 0, cp1 = 0, cp2 = 0, cp3 = 0, ca0 = 0, ca1 = 0, ca2 = 0, ca3 = 0;
    const V cn = p.c[i];
    const unsigned nn = (unsigned)(i - p.n_max);
#pragma unroll
    for (int q = 0; q < PW; ++q) {
      const T x = T(lane * PW + q);
      while (wb < W - 3 && T(base + (wb + 1) * p.R) + gd[(wb + 1) * stride] <= x) ++wb;
      if (wb != cur) {
        cur = wb;
        const T X0 = T(base + (wb - 1) * p.R) + gd[(wb - 1) * stride];
        X1 = T(base + wb * p.R) + gd[wb * stride];
        const T X2 = T(base + (wb + 1) * p.R) + gd[(wb + 1) * stride];
        const T X3 = T(base + (wb + 2) * p.R) + gd[(wb + 2) * stride];
        h21 = X2 - X1;
        h10 = X1 - X0;
        const T r21 = T(1) / h21, r10 = T(1) / h10, r32 = T(1) / (X3 - X2);
        const T r20 = T(1) / (X2 - X0), r31 = T(1) / (X3 - X1), r30 = T(1) / (X3 - X0);
        {
          const T f0 = gph[(wb - 1) * stride], f1 = gph[wb * stride];
          const T f2 = gph[(wb + 1) * stride], f3 = gph[(wb + 2) * stride];
          const T d12 = (f2 - f1) * r21, d01 = (f1 - f0) * r10, d23 = (f3 - f2) * r32;
          const T d012 = (d12 - d01) * r20, d123 = (d23 - d12) * r31;
          cp0 = f1; cp1 = d12; cp2 = d012; cp3 = (d123 - d012) * r30;
        }
        {
          const T f0 = ga[(wb - 1) * stride], f1 = ga[wb * stride];
          const T f2 = ga[(wb + 1) * stride], f3 = ga[(wb + 2) * stride];
          const T d12 = (f2 - f1) * r21, d01 = (f1 - f0) * r10, d23 = (f3 - f2) * r32;
          const T d012 = (d12 - d01) * r20, d123 = (d23 - d12) * r31;
          ca0 = f1; ca1 = d12; ca2 = d012; ca3 = (d123 - d012) * r30;
        }
      }
      const T tau = x - X1;
      const T e2 = tau - h21;
      const T e0 = tau + h10;
      const T phv = cp0 + tau * (cp1 + e2 * (cp2 + e0 * cp3));
      const T av = ca0 + tau * (ca1 + e2 * (ca2 + e0 * ca3));
      const unsigned nm = (nn * (unsigned)(m0 + lane * PW + q)) & mask;
      T t = T(nm) * invN + phv;
      t -= rint(t);
      T sn, cs;
      sincospi_t(T(2) * t, &sn, &cs);
      const T ar = av * cn.x, ai = av * cn.y;
      accr[q] += ar * cs - ai * sn;
      acci[q] += ar * sn + ai * cs;
    }
  }
  V* out = p.part + (long long)group * p.N + m0 + lane * PW;
#pragma unroll
  for (int q = 0; q < PW; ++q) {
    V v;
    v.x = accr[q];
    v.y = acci[q];
    out[q] = v;
  }
}

// ----------------------------------------------------------------------------
// field bookkeeping: partial sums, absorber, reflection, I/O
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_reduce(const ReduceArgs<T> p) {
  using V = typename C2<T>::type;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  auto sum_at = [&](int mm) {
    V s;
    s.x = T(0); s.y = T(0);
    for (int g = 0; g < p.n_part; ++g) {
      const V v = p.part[(long long)g * p.N + mm];
      s.x += v.x; s.y += v.y;
    }
    if (p.W) { const T w = p.W[mm]; s.x *= w; s.y *= w; }
    return s;
  };
  if (!p.mirror) {
    if (m < p.N) p.u[m] = sum_at(m);
    return;
  }
  if (m > p.N / 2) return;
  const int mm = (p.N - m) & (p.N - 1);
  const V a = sum_at(m);
  const V b = (mm == m) ? a : sum_at(mm);
  const T sg = T(p.mirror);
  V ua, ub;
  ua.x = T(0.5) * (a.x + sg * b.x); ua.y = T(0.5) * (a.y + sg * b.y);
  ub.x = T(0.5) * (b.x + sg * a.x); ub.y = T(0.5) * (b.y + sg * a.y);
  p.u[m] = ua;
  p.u[mm] = ub;
}

template <typename T>
__global__ void k_init(const double* __restrict__ u0, int n_z, int N, int mirror,
                       typename C2<T>::type* __restrict__ u) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  typename C2<T>::type v;
  if (!mirror) {
    v.x = T(u0[2 * m]); v.y = T(u0[2 * m + 1]);
  } else if (m >= n_z) {
    v.x = T(u0[2 * (m - n_z)]); v.y = T(u0[2 * (m - n_z) + 1]);
  } else if (m > 0) {
    v.x = T(mirror) * T(u0[2 * (n_z - m)]); v.y = T(mirror) * T(u0[2 * (n_z - m) + 1]);
  } else {
    v.x = T(0); v.y = T(0);
  }
  u[m] = v;
}

template <typename T>
__global__ void k_output(const typename C2<T>::type* __restrict__ u, int offset, int n,
                         double* __restrict__ out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const typename C2<T>::type v = u[offset + m];
  out[2 * m] = double(v.x);
  out[2 * m + 1] = double(v.y);
}

// ----------------------------------------------------------------------------
// (a) pruned DFT: N = N1 N2, n = n1 N2 + n2, k = k1 + N1 k2
//   X[k1 + N1 k2] = sum_n2 w_{N2}^{n2 k2} w_N^{n2 k1} sum_n1 x[n1 N2 + n2] w_{N1}^{n1 k1}
// pass 1 (N1 > 1): one thread per column n2, direct length-N1 DFT + twiddle;
// pass 2: one CTA per row k1, radix-2 Stockham FFT of length N2 in shared
// memory, writes only the kept bins |n| <= n_max as c_n.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename C2<T>::type cmul(typename C2<T>::type a,
                                                     typename C2<T>::type b) {
  typename C2<T>::type r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

template <typename T>
__global__ void k_fft1(const FftArgs<T> p) {
  using V = typename C2<T>::type;
  const int n2 = blockIdx.x * blockDim.x + threadIdx.x;
  if (n2 >= p.N2) return;
  for (int k1 = 0; k1 < p.N1; ++k1) {
    V acc;
    acc.x = T(0); acc.y = T(0);
    for (int n1 = 0; n1 < p.N1; ++n1) {
      const V x = p.u[(long long)n1 * p.N2 + n2];
      const V w = p.tw[(long long)((n1 * k1) % p.N1) * p.N2];
      const V t = cmul<T>(x, w);
      acc.x += t.x; acc.y += t.y;
    }
    p.Y[(long long)k1 * p.N2 + n2] = cmul<T>(acc, p.tw[(long long)n2 * k1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fft2(const FftArgs<T> p) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  V* B = A + p.N2;
  const int k1 = blockIdx.x;
  const V* src = (p.N1 > 1) ? p.Y + (long long)k1 * p.N2 : p.u;
  for (int x = threadIdx.x; x < p.N2; x += blockDim.x) A[x] = src[x];
  __syncthreads();
  const int half = p.N2 >> 1;
  for (int m = 1, lg = 0; m < p.N2; m <<= 1, ++lg) {
    const long long twstep = (long long)p.N >> (lg + 1);   // N / (2m)
    for (int b = threadIdx.x; b < half; b += blockDim.x) {
      const int j = b >> lg;
      const int k = b & (m - 1);
      const V w = p.tw[k * twstep];
      const V c0 = A[k + j * m];
      const V c1 = cmul<T>(w, A[k + j * m + half]);
      V y0, y1;
      y0.x = c0.x + c1.x; y0.y = c0.y + c1.y;
      y1.x = c0.x - c1.x; y1.y = c0.y - c1.y;
      B[k + 2 * j * m] = y0;
      B[k + 2 * j * m + m] = y1;
    }
    __syncthreads();
    V* t = A; A = B; B = t;
  }
  for (int k2 = threadIdx.x; k2 < p.N2; k2 += blockDim.x) {
    const long long b = (long long)k1 + (long long)p.N1 * k2;
    int n;
    if (b <= p.n_max) n = (int)b;
    else if (b >= (long long)p.N - p.n_max) n = (int)(b - p.N);
    else continue;
    V v = A[k2];
    v.x *= p.inv_N; v.y *= p.inv_N;
    p.c[n + p.n_max] = cmul<T>(v, p.ephi[n + p.n_max]);
  }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
template <typename T>
cudaError_t launch_init(const double* u0, int n_z, int N, int mirror, typename C2<T>::type* u,
                        cudaStream_t s) {
  k_init<T><<<(N + 255) / 256, 256, 0, s>>>(u0, n_z, N, mirror, u);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce(const ReduceArgs<T>& a, cudaStream_t s) {
  const int n = a.mirror ? a.N / 2 + 1 : a.N;
  k_reduce<T><<<(n + 255) / 256, 256, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fft(const FftArgs<T>& a, cudaStream_t s) {
  if (a.N1 > 1) {
    k_fft1<T><<<(a.N2 + 127) / 128, 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const size_t smem = 2 * (size_t)a.N2 * sizeof(typename C2<T>::type);
  k_fft2<T><<<a.N1, 256, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_march(const MarchArgs<T>& a, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.M + 31) / 32, (a.NRT + 7) / 8);
  k_march<T><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_bracket(const BracketArgs<T>& a, cudaStream_t s) {
  dim3 grid((a.M + 127) / 128, a.NRT - 1);
  k_bracket<T><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <typename T>
size_t resum_smem_bytes(int wcap, int warps_per_cta) {
  return (size_t)warps_per_cta * 3 * wcap * sizeof(T);
}

template <typename T>
cudaError_t launch_resum(const ResumArgs<T>& a, int warps_per_cta, cudaStream_t s) {
  const int items = a.n_tiles * a.n_groups;
  const int grid = (items + warps_per_cta - 1) / warps_per_cta;
  const size_t smem = resum_smem_bytes<T>(a.wcap, warps_per_cta);
  switch (a.PW) {
    case 2: k_resum<T, 2><<<grid, warps_per_cta * 32, smem, s>>>(a); break;
    case 4: k_resum<T, 4><<<grid, warps_per_cta * 32, smem, s>>>(a); break;
    case 8: k_resum<T, 8><<<grid, warps_per_cta * 32, smem, s>>>(a); break;
    case 16: k_resum<T, 16><<<grid, warps_per_cta * 32, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t prepare_kernels(int resum_smem) {
  cudaError_t e = cudaFuncSetAttribute(k_fft2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(2 * 4096 * sizeof(typename C2<T>::type)));
  if (e != cudaSuccess) return e;
  const void* fs[] = {(const void*)k_resum<T, 2>, (const void*)k_resum<T, 4>,
                      (const void*)k_resum<T, 8>, (const void*)k_resum<T, 16>};
  for (const void* f : fs) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, resum_smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t prepare_fft_kernels() {
  return cudaFuncSetAttribute(k_fft2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(2 * 4096 * sizeof(typename C2<T>::type)));
}

template <typename T>
cudaError_t launch_output(const typename C2<T>::type* u, int offset, int n, double* out,
                          cudaStream_t s) {
  k_output<T><<<(n + 255) / 256, 256, 0, s>>>(u, offset, n, out);
  return cudaGetLastError();
}

#define SWKB_INSTANTIATE(T)                                                                     \
  template cudaError_t launch_init<T>(const double*, int, int, int, C2<T>::type*, cudaStream_t); \
  template cudaError_t launch_reduce<T>(const ReduceArgs<T>&, cudaStream_t);                    \
  template cudaError_t launch_fft<T>(const FftArgs<T>&, cudaStream_t);                          \
  template cudaError_t launch_march<T>(const MarchArgs<T>&, cudaStream_t);                      \
  template cudaError_t launch_bracket<T>(const BracketArgs<T>&, cudaStream_t);                  \
  template cudaError_t launch_resum<T>(const ResumArgs<T>&, int, cudaStream_t);                 \
  template cudaError_t launch_output<T>(const C2<T>::type*, int, int, double*, cudaStream_t);   \
  template size_t resum_smem_bytes<T>(int, int);                                                \
  template cudaError_t prepare_kernels<T>(int);                                                 \
  template cudaError_t prepare_fft_kernels<T>();

SWKB_INSTANTIATE(float)
SWKB_INSTANTIATE(double)

}  // namespace swkb
