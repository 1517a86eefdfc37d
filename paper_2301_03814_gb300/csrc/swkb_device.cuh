// Device bodies of the screened-WKB screen step (sm_103a), templated on the
// arithmetic type T.  Every step is a __device__ function of its (virtual)
// block index and thread index, called by the standalone kernels of
// swkb_kernels.cu (one launch per step) and by the persistent batch kernel of
// swkb_batch.cu (many instances' steps as work items of one launch), so both
// run the same arithmetic.  See swkb_kernels.cu for the step list.
#pragma once

#include <math.h>
#include <stdint.h>

#include <utility>

#include "swkb_internal.h"

namespace swkb {

// ----------------------------------------------------------------------------
// small helpers
// ----------------------------------------------------------------------------
// Bounds-checked builds (-DSWKB_BOUNDS_CHECK, libswkb_checked.so): an index
// outside [0, n) sets ST_BOUNDS in the kernel's status bits, which the host
// reports as an error, and is clamped into range so that the access stays
// inside its buffer.  Plain builds compile the check away.
__device__ __forceinline__ long long bchk(long long i, long long n, unsigned& st) {
#ifdef SWKB_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    st |= ST_BOUNDS;
    return i < 0 ? 0 : n - 1;
  }
#else
  (void)n; (void)st;
#endif
  return i;
}

// Loads of data another kernel (or, in the persistent batch kernel, another
// work item of the same kernel) produced: LD_NC through the read-only
// (non-coherent) path, valid only when nothing writes the data during the
// kernel; LD_CG from L2, bypassing L1, for the persistent kernel, where the
// producer ran on another SM while this kernel was running.
enum { LD_PLAIN = 0, LD_NC = 1, LD_CG = 2 };
template <int LD, typename T>
__device__ __forceinline__ T ld(const T* p) {
  if constexpr (LD == LD_NC) return __ldg(p);
  else if constexpr (LD == LD_CG) return __ldcg(p);
  else return *p;
}

// Barrier over the threads running one virtual block: the whole CTA
// (BAR = 0, the standalone kernels), or one 128-thread half of it (BAR = 1:
// named barrier 1 + sub, the persistent kernel runs two such blocks per CTA).
template <int BAR>
__device__ __forceinline__ void vb_sync(int sub) {
  if constexpr (BAR == 0) {
    (void)sub;
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + sub) : "memory");
  }
}

// sin / cos of 2 pi t for |t| <= 1/2: the FP32 path uses the special-function
// unit (absolute error ~2^-21 on [-pi, pi]); the FP64 path stays exact.
__device__ __forceinline__ void sincos_turns(float t, float* s, float* c) {
  __sincosf(6.28318530717958647692f * t, s, c);
}
__device__ __forceinline__ void sincos_turns(double t, double* s, double* c) {
  sincospi(2.0 * t, s, c);
}

// Exact integer/float steps of the resummation kept off the conversion units
// in FP32: floor of |y| < 2^22 by a round-down add of 1.5 * 2^23, the float
// of an integer k < 2^23 from its bits, and t - rint(t) for |t| < 2^22 by
// adding and subtracting 1.5 * 2^23 (round to nearest even, as rint).  The
// FP64 versions are the plain operations.
__device__ __forceinline__ int ifloor_small(float y) {
  return (int)(__float_as_uint(__fadd_rd(y, 12582912.f)) - 0x4B400000u);
}
__device__ __forceinline__ int ifloor_small(double y) { return (int)floor(y); }
__device__ __forceinline__ float exact_u2f(unsigned k, float) {
  return __uint_as_float(0x4B000000u | k) - 8388608.f;
}
__device__ __forceinline__ double exact_u2f(unsigned k, double) { return (double)k; }
__device__ __forceinline__ float minus_rint(float t) {
  const float r = (t + 12582912.f) - 12582912.f;
  return t - r;
}
__device__ __forceinline__ double minus_rint(double t) { return t - rint(t); }

// 1/sqrt: FP32 via the special-function unit (2 ulp), FP64 correctly-rounded
// to 1 ulp.  Small-quotient division: FP32 fast (2 ulp), FP64 IEEE.
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }
__device__ __forceinline__ float fdiv_t(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_t(double a, double b) { return a / b; }

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
  // outside [0, n_int] (or NaN): flag; the interval index is clamped in
  // integers (a flagged ray's values are discarded, its reads stay in bounds)
  if (!(u >= T(0) && u <= T(m.n_int))) st |= ST_RANGE;
  const int i = min(max((int)floor(u), 0), m.n_int - 1);
  const T t = u - T(i);
  T a0, a1, a2, a3, a4, a5;
  load6<T>(m.coef + bchk((long long)c * m.col_stride + (long long)i * 8, m.size - 7, st), a0, a1,
           a2, a3, a4, a5);
  // Horner with derivatives (synthetic division): p, p', p''/2 at t
  T b = a5 * t + a4;                                     // coefficient 4
  T d2 = a5;                                             // coefficient 3
  T d1 = a5 * t + b;
  b = b * t + a3;
  d2 = d2 * t + d1; d1 = d1 * t + b; b = b * t + a2;     // coefficient 2
  d2 = d2 * t + d1; d1 = d1 * t + b; b = b * t + a1;     // coefficient 1
  d2 = d2 * t + d1; d1 = d1 * t + b; b = b * t + a0;     // coefficient 0
  e = b;
  ez = d1 * m.inv_h;
  ezz = d2 * m.inv_h2;   // inv_h2 = 2 / h^2
}

// eps - eps_ref, eps_z, eps_zz at RK4 stage l and height z.  MULTI: the
// profile has several range columns (else column 0 everywhere).
template <typename T, bool MULTI>
__device__ __forceinline__ void medium_eval(const MarchArgs<T>& p, int l, T z, T& e, T& ez,
                                            T& ezz, unsigned& st) {
  T zz = z, sg = T(1);
  if (p.med.mirrored) {
    const T d = z - p.med.z_mirror;
    sg = d < T(0) ? T(-1) : T(1);
    zz = p.med.z_mirror + fabs(d);
  }
  if (!MULTI) {
    col_eval(p.med, 0, zz, e, ez, ezz, st);
  } else {
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
template <typename T, bool MULTI>
__device__ __forceinline__ Ray<T> rhs(const MarchArgs<T>& p, int l, T s, T kap, T pb, T pb2,
                                      const Ray<T>& y, unsigned& st) {
  T e, ez, ezz;
  medium_eval<T, MULTI>(p, l, s + y.dz, e, ez, ezz, st);
  const T Q = kap + y.dQ;
  const T D = e - y.dQ * (T(2) * kap + y.dQ);
  T P2 = pb2 + D;
  if (!(P2 > T(0))) { st |= ST_TURNING; P2 = pb2; }
  if (!(y.Zs > T(0))) st |= ST_CAUSTIC;
  const T iP = rsqrt_t(P2);
  const T P = P2 * iP;
  Ray<T> d;
  d.dz = Q * iP;
  d.dQ = T(0.5) * ez * iP;
  d.rh = (e - kap * y.dQ - pb * fdiv_t(D, pb + P)) * iP;
  const T PsiP = (ez * y.Zs - T(2) * Q * y.Qs) * (T(0.5) * iP * iP);   // P_s / P
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
template <typename T, bool MULTI, bool PLANES>
__device__ __forceinline__ void march_body(const MarchArgs<T>& p, int bx, int by, int tx, int ty) {
  const int r = bx * 32 + tx;       // marched mode (output column)
  const int j = by * 8 + ty;
  if (r >= p.Mr || j >= p.NRT) return;
  unsigned st = 0;
  const int i = r + p.mode_off;
  const T kap = p.kappa[i], pb = p.pbar[i], pb2 = p.pbar2[i];
  const T s = p.z_lo + T((j - p.G) * p.R) * p.dz;
  T e, ez, ezz;
  medium_eval<T, MULTI>(p, 0, s, e, ez, ezz, st);
  T P0sq = pb2 + e;
  if (!(P0sq > T(0))) { st |= ST_TURNING; P0sq = pb2; }
  const T P0 = sqrt(P0sq);
  Ray<T> y{T(0), T(0), T(0), T(1), T(0)};
  const T h = p.h, hh = T(0.5) * p.h, h6 = p.h / T(6);
  // landing quantities at RK4 stage l (the screen's end, or a plane inside it)
  auto land = [&](int l, T* od, T* oph, T* oa) {
    const long long o = bchk((long long)j * p.Mr + r, (long long)p.NRT * p.Mr, st);
    if (!(y.Zs > T(0))) st |= ST_CAUSTIC;
    T e1, ez1, ezz1;
    medium_eval<T, MULTI>(p, l, s + y.dz, e1, ez1, ezz1, st);
    T P1sq = pb2 + e1 - y.dQ * (T(2) * kap + y.dQ);
    if (!(P1sq > T(0))) { st |= ST_TURNING; P1sq = pb2; }
    const T Zs = y.Zs > T(0) ? y.Zs : T(1);
    od[o] = y.dz * p.inv_dz;
    oph[o] = y.rh * p.k_over_2pi;
    oa[o] = sqrt(P0 * rsqrt_t(P1sq) / Zs);
  };
  for (int n = 0; n < p.Nt; ++n) {
    const Ray<T> k1 = rhs<T, MULTI>(p, 2 * n, s, kap, pb, pb2, y, st);
    const Ray<T> k2 = rhs<T, MULTI>(p, 2 * n + 1, s, kap, pb, pb2, axpy(y, hh, k1), st);
    const Ray<T> k3 = rhs<T, MULTI>(p, 2 * n + 1, s, kap, pb, pb2, axpy(y, hh, k2), st);
    const Ray<T> k4 = rhs<T, MULTI>(p, 2 * n + 2, s, kap, pb, pb2, axpy(y, h, k3), st);
    y.dz += h6 * (k1.dz + T(2) * k2.dz + T(2) * k3.dz + k4.dz);
    y.dQ += h6 * (k1.dQ + T(2) * k2.dQ + T(2) * k3.dQ + k4.dQ);
    y.rh += h6 * (k1.rh + T(2) * k2.rh + T(2) * k3.rh + k4.rh);
    y.Zs += h6 * (k1.Zs + T(2) * k2.Zs + T(2) * k3.Zs + k4.Zs);
    y.Qs += h6 * (k1.Qs + T(2) * k2.Qs + T(2) * k3.Qs + k4.Qs);
    if (PLANES && (n + 1) % p.plane_steps == 0 && n + 1 < p.Nt) {
      const long long po = (long long)((n + 1) / p.plane_steps - 1) * p.NRT * p.Mr;
      land(2 * (n + 1), p.pl_d + po, p.pl_ph + po, p.pl_a + po);
    }
  }
  land(2 * p.Nt, p.out_d, p.out_ph, p.out_a);
  if (st) atomicOr(p.status, st);
}

template <typename T, bool MULTI, bool PLANES>
__global__ void __launch_bounds__(256) k_march(const MarchArgs<T> p) {
  march_body<T, MULTI, PLANES>(p, blockIdx.x, blockIdx.y, threadIdx.x, threadIdx.y);
}

// ----------------------------------------------------------------------------
// (b) ray march, FP32 path with packed f32x2 arithmetic: each thread marches
// two rays of one mode (see k_march_x2 for which).  The medium lookups stay per ray; the
// right-hand side of the ray + variational system and the RK4 updates run on
// register pairs, halving their issue slots (same IEEE round-to-nearest
// operations as the scalar kernel, in the same order up to FMA contraction).
// ----------------------------------------------------------------------------
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 mk2(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void sp2(f2 x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x.v));
}
__device__ __forceinline__ f2 bc2(float a) { return mk2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
  f2 r;
  asm("add.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
  f2 r;
  asm("sub.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
  f2 r;
  asm("mul.rn.ftz.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {   // a b + c
  f2 r;
  asm("fma.rn.ftz.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

struct Ray2 {
  f2 dz, dQ, rh, Zs, Qs;
};

// FP32 medium lookup at table position u (intervals from the table origin;
// the table stores the reflection, so there is no mirror step).  Returns
// p(t), p'(t) and p''(t)/2 of the interval's quintic (derivatives in t).
// u outside [0, top] or NaN flags ST_RANGE and is evaluated at the clamped
// position.  floor(u) comes from one round-down add of 1.5 * 2^23 (exact for
// 0 <= u < 2^22), keeping the conversion units free.
__device__ __forceinline__ void horner5(const float* q, float t, float& e, float& d1, float& d2) {
  float a0, a1, a2, a3, a4, a5;
  load6<float>(q, a0, a1, a2, a3, a4, a5);
  float b = a5 * t + a4;
  float c2 = a5;
  float c1 = a5 * t + b;
  b = b * t + a3;
  c2 = c2 * t + c1; c1 = c1 * t + b; b = b * t + a2;
  c2 = c2 * t + c1; c1 = c1 * t + b; b = b * t + a1;
  c2 = c2 * t + c1; c1 = c1 * t + b; b = b * t + a0;
  e = b; d1 = c1; d2 = c2;
}

// Cubic piece b0..b3 in tau (one 16-byte load): value, first derivative and
// half the second derivative by synthetic division (6 FMAs).
__device__ __forceinline__ void horner3(const float* q, float t, float& e, float& d1, float& d2) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(q));
  float b = v.w * t + v.z;
  float c1 = v.w * t + b;
  b = b * t + v.y;
  const float c2 = v.w * t + c1;
  c1 = c1 * t + b;
  b = b * t + v.x;
  e = b; d1 = c1; d2 = c2;
}

template <bool CUBIC>
__device__ __forceinline__ void table_eval(const float* q, float t, float& e, float& d1,
                                           float& d2) {
  if (CUBIC) horner3(q, t, e, d1, d2);
  else horner5(q, t, e, d1, d2);
}

// CUBIC: the table holds cubic pieces (4 slots each, u in piece units).
template <bool MULTI, bool CUBIC>
__device__ __forceinline__ void med32(const MarchArgs<float>& p, int l, float u, float& e,
                                      float& d1, float& d2, unsigned& st) {
  constexpr int W = CUBIC ? 4 : 8;
  const float uc = fminf(fmaxf(u, 0.f), p.med.top);
  if (uc != u) st |= ST_RANGE;
  const float v = __fadd_rd(uc, 12582912.f);
  const int i = (int)(__float_as_uint(v) - 0x4B400000u);
  const float t = uc - (v - 12582912.f);
  if (!MULTI) {
    table_eval<CUBIC>(p.med.coef + bchk((long long)i * W, p.med.size - (W - 1), st), t, e, d1, d2);
  } else {
    const int c = __ldg(p.st.c + l);
    const float th = __ldg(p.st.th + l);
    const float* q = p.med.coef + bchk((long long)c * p.med.col_stride + (long long)i * W,
                                       p.med.size - (th == 0.f ? W - 1 : p.med.col_stride + W - 1),
                                       st);
    if (th == 0.f) {
      table_eval<CUBIC>(q, t, e, d1, d2);
    } else if (th == 1.f) {
      table_eval<CUBIC>(q + p.med.col_stride, t, e, d1, d2);
    } else {
      float e0, e1, f0, f1, g0, g1;
      table_eval<CUBIC>(q, t, e0, f0, g0);
      table_eval<CUBIC>(q + p.med.col_stride, t, e1, f1, g1);
      e = (1.f - th) * e0 + th * e1;
      d1 = (1.f - th) * f0 + th * f1;
      d2 = (1.f - th) * g0 + th * g1;
    }
  }
}

// x-form right-hand side for two rays; u2 = their table positions.  With
// he = eps_z / 2 and hee = eps_zz / 2 (table derivatives times 1 / (2 h) and
// 1 / h^2):  z' = Q/P,  Q' = he/P,  r' - P_bar as in the scalar kernel,
//   -P_s/P = (Q Q_s - he Z_s)/P^2,  Z_s' = (Q_s + Q (-P_s/P))/P,
//   Q_s' = (hee Z_s + he (-P_s/P))/P.
template <bool MULTI, bool CUBIC>
__device__ __forceinline__ Ray2 rhs2(const MarchArgs<float>& p, int l, f2 u2, f2 kap, f2 m2kap,
                                     f2 mkap, f2 pb, f2 mpb, float pb2, f2 pb2v, f2 ihh,
                                     f2 mihh, f2 ihq, const Ray2& y, unsigned& st, float& mnP,
                                     float& mnZ) {
  float ua, ub;
  sp2(u2, ua, ub);
  float ea, d1a, d2a, eb, d1b, d2b;
  med32<MULTI, CUBIC>(p, l, ua, ea, d1a, d2a, st);
  med32<MULTI, CUBIC>(p, l, ub, eb, d1b, d2b, st);
  const f2 e = mk2(ea, eb), d1 = mk2(d1a, d1b);
  const f2 he = mul2(d1, ihh), mhe = mul2(d1, mihh), hee = mul2(mk2(d2a, d2b), ihq);
  const f2 Q = add2(kap, y.dQ);
  const f2 D = fma2(y.dQ, sub2(m2kap, y.dQ), e);           // e - dQ (2 kappa + dQ)
  float P2a, P2b;
  sp2(add2(pb2v, D), P2a, P2b);
  // Turning points (P^2 <= 0) and caustics (Z_s <= 0) at any stage: running
  // minima, checked once after the march (a ray that meets one goes on with
  // NaN values; its table positions are clamped, its status is an error).
  float Zsa, Zsb;
  sp2(y.Zs, Zsa, Zsb);
  mnP = fminf(mnP, fminf(P2a, P2b));
  mnZ = fminf(mnZ, fminf(Zsa, Zsb));
  (void)pb2;
  const float iPa = rsqrtf(P2a), iPb = rsqrtf(P2b);
  const f2 iP = mk2(iPa, iPb);
  const f2 P = mul2(mk2(P2a, P2b), iP);
  float da, db;
  sp2(add2(pb, P), da, db);
  const f2 rden = mk2(__fdividef(1.f, da), __fdividef(1.f, db));
  Ray2 d;
  d.dz = mul2(Q, iP);
  d.dQ = mul2(he, iP);
  // (e - kappa dQ - P_bar D / (P_bar + P)) / P
  d.rh = mul2(fma2(mpb, mul2(D, rden), fma2(mkap, y.dQ, e)), iP);
  const f2 mPsiP = mul2(fma2(mhe, y.Zs, mul2(Q, y.Qs)), mul2(iP, iP));
  d.Zs = mul2(fma2(Q, mPsiP, y.Qs), iP);
  d.Qs = mul2(fma2(he, mPsiP, mul2(hee, y.Zs)), iP);
  return d;
}

__device__ __forceinline__ Ray2 axpy2(const Ray2& y, f2 a, const Ray2& k) {
  return Ray2{fma2(a, k.dz, y.dz), fma2(a, k.dQ, y.dQ), fma2(a, k.rh, y.rh), fma2(a, k.Zs, y.Zs),
              fma2(a, k.Qs, y.Qs)};
}

// Thread t marches rays q and q + NH of mode r, t = q Mr + r (NH = ceil(NRT / 2)):
// a warp's lanes are consecutive modes at one launch height (their table
// reads stay within a few intervals) and no lane idles at the end of a row.
template <bool MULTI, bool PLANES, bool CUBIC>
__device__ __forceinline__ void march_x2_body(const MarchArgs<float>& p, int blk, int tid) {
  const int NH = (p.NRT + 1) >> 1;
  const int t = blk * 256 + tid;
  if (t >= p.Mr * NH) return;
  const int ja = t / p.Mr;
  const int r = t - ja * p.Mr;
  const int jb = ja + NH;
  const bool has_b = jb < p.NRT;
  unsigned st = 0;
  const int i = r + p.mode_off;
  const float kap = p.kappa[i], pb = p.pbar[i], pb2 = p.pbar2[i];
  // launch heights in table intervals
  const float ua = fmaf(float((ja - p.G) * p.R), p.u_dz, p.u_lo);
  const float ub = has_b ? fmaf(float((jb - p.G) * p.R), p.u_dz, p.u_lo) : ua;
  const f2 s = mk2(ua, ub), kv = bc2(kap), m2kap = bc2(-2.f * kap), mkap = bc2(-kap);
  const f2 pbv = bc2(pb), mpb = bc2(-pb), pb2v = bc2(pb2);
  const float ihs = p.med.inv_h;
  const f2 ih = bc2(ihs), ihh = bc2(0.5f * ihs), mihh = bc2(-0.5f * ihs);
  const f2 ihq = bc2(0.5f * p.med.inv_h2);   // inv_h2 = 2 / h^2
  float e0a, e0b, t0, t1;
  med32<MULTI, CUBIC>(p, 0, ua, e0a, t0, t1, st);
  med32<MULTI, CUBIC>(p, 0, ub, e0b, t0, t1, st);
  float P0a = pb2 + e0a, P0b = pb2 + e0b;
  if (!(P0a > 0.f)) { st |= ST_TURNING; P0a = pb2; }
  if (!(P0b > 0.f)) { st |= ST_TURNING; P0b = pb2; }
  P0a = sqrtf(P0a);
  P0b = sqrtf(P0b);
  const f2 zero = bc2(0.f);
  Ray2 y{zero, zero, zero, bc2(1.f), zero};
  const f2 h = bc2(p.h), hh = bc2(0.5f * p.h), h6 = bc2(p.h / 6.f);
  // table position of a ray: launch position + dz / h_table
  const auto pos = [&](const Ray2& w) { return fma2(w.dz, ih, s); };
  // landing quantities at RK4 stage l (the screen's end, or a plane inside it)
  const auto land = [&](int l, float* od, float* oph, float* oam) {
    const long long nrm = (long long)p.NRT * p.Mr;
    const long long oa = bchk((long long)ja * p.Mr + r, nrm, st);
    const long long ob = has_b ? bchk((long long)jb * p.Mr + r, nrm, st) : oa;
    float dza, dzb, dQa, dQb, rha, rhb, Zsa, Zsb, u1a, u1b;
    sp2(y.dz, dza, dzb);
    sp2(y.dQ, dQa, dQb);
    sp2(y.rh, rha, rhb);
    sp2(y.Zs, Zsa, Zsb);
    sp2(pos(y), u1a, u1b);
    if (!(Zsa > 0.f) || !(Zsb > 0.f)) st |= ST_CAUSTIC;
    float e1a, e1b, s0, s1;
    med32<MULTI, CUBIC>(p, l, u1a, e1a, s0, s1, st);
    med32<MULTI, CUBIC>(p, l, u1b, e1b, s0, s1, st);
    float P1a = pb2 + e1a - dQa * (2.f * kap + dQa);
    float P1b = pb2 + e1b - dQb * (2.f * kap + dQb);
    if (!(P1a > 0.f)) { st |= ST_TURNING; P1a = pb2; }
    if (!(P1b > 0.f)) { st |= ST_TURNING; P1b = pb2; }
    const float Za = Zsa > 0.f ? Zsa : 1.f, Zb = Zsb > 0.f ? Zsb : 1.f;
    od[oa] = dza * p.inv_dz;
    oph[oa] = rha * p.k_over_2pi;
    oam[oa] = sqrtf(P0a * rsqrtf(P1a) / Za);
    if (has_b) {
      od[ob] = dzb * p.inv_dz;
      oph[ob] = rhb * p.k_over_2pi;
      oam[ob] = sqrtf(P0b * rsqrtf(P1b) / Zb);
    }
  };
  // RK4: y + h/6 k1 + h/3 k2 + h/3 k3 + h/6 k4, accumulated as the stages
  // complete (k1..k3 need not stay live)
  const f2 h3 = bc2(p.h / 3.f);
  float mnP = 1.f, mnZ = 1.f;   // smallest P^2 and Z_s met (1: none below)
  for (int n = 0; n < p.Nt; ++n) {
    const Ray2 k1 = rhs2<MULTI, CUBIC>(p, 2 * n, pos(y), kv, m2kap, mkap, pbv, mpb, pb2, pb2v, ihh,
                                mihh, ihq, y, st, mnP, mnZ);
    Ray2 acc = axpy2(y, h6, k1);
    const Ray2 y2 = axpy2(y, hh, k1);
    const Ray2 k2 = rhs2<MULTI, CUBIC>(p, 2 * n + 1, pos(y2), kv, m2kap, mkap, pbv, mpb, pb2, pb2v,
                                ihh, mihh, ihq, y2, st, mnP, mnZ);
    acc = axpy2(acc, h3, k2);
    const Ray2 y3 = axpy2(y, hh, k2);
    const Ray2 k3 = rhs2<MULTI, CUBIC>(p, 2 * n + 1, pos(y3), kv, m2kap, mkap, pbv, mpb, pb2, pb2v,
                                ihh, mihh, ihq, y3, st, mnP, mnZ);
    acc = axpy2(acc, h3, k3);
    const Ray2 y4 = axpy2(y, h, k3);
    const Ray2 k4 = rhs2<MULTI, CUBIC>(p, 2 * n + 2, pos(y4), kv, m2kap, mkap, pbv, mpb, pb2, pb2v,
                                ihh, mihh, ihq, y4, st, mnP, mnZ);
    y = axpy2(acc, h6, k4);
    if (PLANES && (n + 1) % p.plane_steps == 0 && n + 1 < p.Nt) {
      const long long po = (long long)((n + 1) / p.plane_steps - 1) * p.NRT * p.Mr;
      land(2 * (n + 1), p.pl_d + po, p.pl_ph + po, p.pl_a + po);
    }
  }
  land(2 * p.Nt, p.out_d, p.out_ph, p.out_a);
  if (!(mnP > 0.f)) st |= ST_TURNING;
  if (!(mnZ > 0.f)) st |= ST_CAUSTIC;
  if (st) atomicOr(p.status, st);
}

// 4 CTAs of 256 threads per SM (64 registers)
template <bool MULTI, bool PLANES, bool CUBIC>
__global__ void __launch_bounds__(256, 4) k_march_x2(const MarchArgs<float> p) {
  march_x2_body<MULTI, PLANES, CUBIC>(p, blockIdx.x, threadIdx.x);
}

// ----------------------------------------------------------------------------
// landing checks and tile brackets
// ----------------------------------------------------------------------------
// Landing of ray j in grid units: g_j = (j - G) R + d_j.  Tile t starts at
// grid point t TM; jlo[t][i] = the j with g_j <= t TM < g_{j+1}.
// One landing pair (j, j + 1) of column i: order and coverage checks, and
// the tile starts the pair brackets.  Returns status bits.
template <typename T>
__device__ __forceinline__ unsigned bracket_pair(const BracketArgs<T>& p, int i, int j, T d0,
                                                 T d1) {
  const int b0 = (j - p.G) * p.R;   // |b0| <= N + G R < 2^31
  const int b1 = b0 + p.R;
  unsigned st = 0;
  if (!(T(p.R) + d1 - d0 > T(0))) st |= ST_CAUSTIC;              // g_{j+1} > g_j
  if (j == 1 && !(d0 <= T(-b0))) st |= ST_COVER;                  // g_1 <= 0
  if (j + 1 == p.NRT - 2 && !(d1 > T(p.N - b1))) st |= ST_COVER;  // g_{NRT-2} > N
  if (p.sym) {   // the mirror family g'_{j'} = N - g_{NRT-j'} must cover too
    if (j == 2 && !(d0 < T(-b0))) st |= ST_COVER;                 // g_2 < 0
    if (j + 1 == p.NRT - 1 && !(d1 >= T(p.N - b1))) st |= ST_COVER;  // g_{NRT-1} >= N
  }
  if (st) return st;
  const int TM = p.TM;
  const float inv_tm = 1.0f / (float)TM;   // exact (TM is a power of two)
  // Both families bracket a tile start only if a multiple of TM lies in
  // [g_j, g_{j+1}] (the mirror family's starts N - t TM are multiples of TM
  // too).  Float estimate with a margin of TM / 1000, far above its rounding;
  // the exact tests below decide the pairs that pass.
  {
    const float g0 = (float)b0 + (float)d0, g1 = (float)b1 + (float)d1;
    if (floorf(g1 * inv_tm + 1e-3f) < ceilf(g0 * inv_tm - 1e-3f)) return 0;
  }
  {
    // tile starts t TM in [g_j, g_{j+1})
    int t0 = (int)ceilf(((float)b0 + (float)d0) * inv_tm);
    int t1 = (int)ceilf(((float)b1 + (float)d1) * inv_tm) - 1;
    t0 = min(max(t0, -1), p.n_tiles + 1);
    t1 = min(max(t1, -1), p.n_tiles + 1);
    for (int k = 0; k < 4 && d0 <= T((t0 - 1) * TM - b0); ++k) --t0;
    for (int k = 0; k < 4 && !(d0 <= T(t0 * TM - b0)); ++k) ++t0;
    for (int k = 0; k < 4 && !(T(t1 * TM - b1) < d1); ++k) --t1;
    for (int k = 0; k < 4 && T((t1 + 1) * TM - b1) < d1; ++k) ++t1;
    t0 = max(t0, 0);
    t1 = min(t1, p.n_tiles);
    for (int t = t0; t <= t1; ++t)
      p.jlo[bchk((long long)t * p.Mr + i, (long long)(p.n_tiles + 1) * p.Mr, st)] = j;
  }
  if (p.sym) {
    // mirror family: its bracket of tile start t TM is ray NRT - 1 - j when
    // g_j < N - t TM <= g_{j+1}
    int t0 = (int)ceilf(((float)p.N - (float)b1 - (float)d1) * inv_tm);
    int t1 = (int)ceilf(((float)p.N - (float)b0 - (float)d0) * inv_tm) - 1;
    t0 = min(max(t0, -1), p.n_tiles + 1);
    t1 = min(max(t1, -1), p.n_tiles + 1);
    // t0 = min t with N - t TM <= g_{j+1};  t1 = max t with g_j < N - t TM
    for (int k = 0; k < 4 && T(p.N - (t0 - 1) * TM - b1) <= d1; ++k) --t0;
    for (int k = 0; k < 4 && !(T(p.N - t0 * TM - b1) <= d1); ++k) ++t0;
    for (int k = 0; k < 4 && !(d0 < T(p.N - t1 * TM - b0)); ++k) --t1;
    for (int k = 0; k < 4 && d0 < T(p.N - (t1 + 1) * TM - b0); ++k) ++t1;
    t0 = max(t0, 0);
    t1 = min(t1, p.n_tiles);
    for (int t = t0; t <= t1; ++t)
      p.jlo_neg[bchk((long long)t * p.Mr + i, (long long)(p.n_tiles + 1) * p.Mr, st)] =
          p.NRT - 1 - j;
  }
  return st;
}

// One thread per landing pair (measured faster than longer per-thread runs:
// the kernel is latency-bound and wants the parallelism).
constexpr int BRACKET_RUN = 1;

template <typename T, int LD>
__device__ __forceinline__ void bracket_body(const BracketArgs<T>& p, int bx, int by, int tid) {
  const int i = bx * 256 + tid;
  const int j0 = by * BRACKET_RUN;
  if (i >= p.Mr) return;
  const int j1 = min(j0 + BRACKET_RUN, p.NRT - 1);   // pairs (j, j + 1), j < j1
  unsigned st = 0;
  unsigned bst = 0;
  const long long nrm = (long long)p.NRT * p.Mr;
  T d0 = ld<LD>(p.d + bchk((long long)j0 * p.Mr + i, nrm, bst));
  for (int j = j0; j < j1; ++j) {
    const T d1 = ld<LD>(p.d + bchk((long long)(j + 1) * p.Mr + i, nrm, bst));
    st |= bracket_pair(p, i, j, d0, d1);
    d0 = d1;
  }
  st |= bst;
  if (st) atomicOr(p.status, st);
}

// Rows of landing pairs beyond the grid's y extent (65535) are taken in
// strides of gridDim.y.
template <typename T>
__global__ void __launch_bounds__(256) k_bracket(const BracketArgs<T> p) {
  const int rows = (p.NRT - 1 + BRACKET_RUN - 1) / BRACKET_RUN;
  for (int by = blockIdx.y; by < rows; by += gridDim.y)
    bracket_body<T, LD_PLAIN>(p, blockIdx.x, by, threadIdx.x);
}

// ----------------------------------------------------------------------------
// (c) + (d) interpolation fused with the modal sum
// ----------------------------------------------------------------------------
// A CTA owns one tile of TM = 32 PW consecutive grid points and one mode
// group; its RESUM_WARPS warps take the group's modes round-robin, each
// summing into registers (lane l holds points l PW .. l PW + PW - 1), and the CTA
// adds the warps' sums in a fixed order before writing one partial per
// (group, point).
//
// Per mode a warp
//  (1) stages the rays landing on the tile -- brackets jlo[t] .. jlo[t+1]
//      with stencil -1 / +2 -- in shared memory: landing X (grid units from
//      the tile start), phase, amplitude;
//  (2) one lane per interval [X_w, X_{w+1}): builds the 4-point Lagrange
//      polynomial through X_{w-1} .. X_{w+2} (Newton form, then monomial in
//      tau = x - X_w) for phase and amplitude into a shared-memory row;
//  (3) every lane evaluates its points: interval lookup (guessed from the
//      mean landing spacing, corrected by comparisons), two cubics, the
//      phase with its integer part exact (k kappa_n (z_m - z_lo) =
//      2 pi (n m mod N) / N), sincos, complex multiply-accumulate.
constexpr int RESUM_WARPS = 4;
constexpr int RESUM_CF = 12;      // X_w, 4 phase + 4 amplitude coefficients, X_{w+1}, 2 pad

template <typename T>
__device__ __forceinline__ int resum_warp_bytes(int wcap) {
  return ((RESUM_CF + 3) * wcap * (int)sizeof(T) + 15) & ~15;
}

// one coefficient row (X_w, phase b0..b3, amplitude a0..a3), vector stores:
// rows are 48 B (FP32) apart, so a quarter-warp writes 32 distinct banks
// Row of interval w: X_w, phase cubic b0..b3, amplitude cubic a0..a3, X_{w+1}.
__device__ __forceinline__ void store_cf(float* p, float X1, float X2, float b0, float b1,
                                         float b2, float b3, float a0, float a1, float a2,
                                         float a3) {
  *reinterpret_cast<float4*>(p) = make_float4(X1, b0, b1, b2);
  *reinterpret_cast<float4*>(p + 4) = make_float4(b3, a0, a1, a2);
  *reinterpret_cast<float4*>(p + 8) = make_float4(a3, X2, 0.f, 0.f);
}
__device__ __forceinline__ void store_cf(double* p, double X1, double X2, double b0, double b1,
                                         double b2, double b3, double a0, double a1, double a2,
                                         double a3) {
  *reinterpret_cast<double2*>(p) = make_double2(X1, b0);
  *reinterpret_cast<double2*>(p + 2) = make_double2(b1, b2);
  *reinterpret_cast<double2*>(p + 4) = make_double2(b3, a0);
  *reinterpret_cast<double2*>(p + 6) = make_double2(a1, a2);
  *reinterpret_cast<double2*>(p + 8) = make_double2(a3, X2);
}

template <typename T>
__device__ __forceinline__ void load_cf(const T* p, T& X1, T& X2, T& b0, T& b1, T& b2, T& b3,
                                        T& a0, T& a1, T& a2, T& a3);
template <>
__device__ __forceinline__ void load_cf<float>(const float* p, float& X1, float& X2, float& b0,
                                               float& b1, float& b2, float& b3, float& a0,
                                               float& a1, float& a2, float& a3) {
  const float4 u = *reinterpret_cast<const float4*>(p);
  const float4 v = *reinterpret_cast<const float4*>(p + 4);
  const float2 w = *reinterpret_cast<const float2*>(p + 8);
  X1 = u.x; b0 = u.y; b1 = u.z; b2 = u.w; b3 = v.x; a0 = v.y; a1 = v.z; a2 = v.w;
  a3 = w.x; X2 = w.y;
}
template <>
__device__ __forceinline__ void load_cf<double>(const double* p, double& X1, double& X2,
                                                double& b0, double& b1, double& b2, double& b3,
                                                double& a0, double& a1, double& a2,
                                                double& a3) {
  const double2 u = *reinterpret_cast<const double2*>(p);
  const double2 v = *reinterpret_cast<const double2*>(p + 2);
  const double2 w = *reinterpret_cast<const double2*>(p + 4);
  const double2 x = *reinterpret_cast<const double2*>(p + 6);
  const double2 y = *reinterpret_cast<const double2*>(p + 8);
  X1 = u.x; b0 = u.y; b1 = v.x; b2 = v.y; b3 = w.x; a0 = w.y; a1 = x.x; a2 = x.y;
  a3 = y.x; X2 = y.y;
}

// Newton divided differences through (X1, X2, X0, X3), rewritten as a cubic
// in tau = x - X1:  b0 + b1 tau + b2 tau^2 + b3 tau^3.
template <typename T>
__device__ __forceinline__ void cubic_through(T f0, T f1, T f2, T f3, T r21, T r10, T r32, T r20,
                                              T r31, T r30, T h21, T h10, T& b0, T& b1, T& b2,
                                              T& b3) {
  const T d12 = (f2 - f1) * r21, d01 = (f1 - f0) * r10, d23 = (f3 - f2) * r32;
  const T d012 = (d12 - d01) * r20, d123 = (d23 - d12) * r31;
  const T d0123 = (d123 - d012) * r30;
  b0 = f1;
  b1 = d12 - h21 * (d012 + d0123 * h10);
  b2 = d012 + d0123 * (h10 - h21);
  b3 = d0123;
}

// One resummation block: blk its index in the launch, tid its thread index
// (0 .. 32 RESUM_WARPS - 1), smem_raw its shared memory (resum_smem_bytes),
// sub the virtual-block slot for the barrier (BAR).
template <typename T, int PW, int LD, int BAR>
__device__ __forceinline__ void resum_body(const ResumArgs<T>& p, int blk, int tid,
                                           unsigned char* smem_raw, int sub) {
  using V = typename C2<T>::type;
  constexpr int LDC = LD == LD_NC ? LD_PLAIN : LD;   // mode coefficients
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int tt = blk % p.n_tiles_run;
  const int group = blk / p.n_tiles_run;
  const int half = p.n_tiles >> 1;
  const int tile = p.sym ? (tt < half ? half + tt : 0) : tt;
  const int wcap = p.wcap;
  const int TM = p.TM;
  unsigned char* wbase = smem_raw + (long long)warp * resum_warp_bytes<T>(wcap);
  T* s_cf = reinterpret_cast<T*>(wbase);            // [wcap][RESUM_CF], 16-byte aligned
  T* s_X = s_cf + RESUM_CF * wcap;
  T* s_ph = s_X + wcap;
  T* s_a = s_ph + wcap;
  const int m0 = tile * TM;
  const int i0 = group * p.modes_per_group;
  const int i1 = min(p.M, i0 + p.modes_per_group);
  const int lgN = __ffs(p.N) - 1;
  const T invN = scalbn(T(1), -lgN);               // exact
  const unsigned mask = (unsigned)p.N - 1u;
  unsigned st = 0;

  T accr[PW], acci[PW];
#pragma unroll
  for (int q = 0; q < PW; ++q) { accr[q] = T(0); acci[q] = T(0); }

  // Software pipeline over this warp's modes: the bracket entries are
  // loaded two modes ahead and the ray window (landing offset, phase,
  // amplitude; the first 32 rays) one mode ahead into registers, so their
  // global-memory latency overlaps the current mode's arithmetic.
  // grounded: mode n < 0 is the mirror image of mode -n (column -n); its
  // ray j' is ray NRT - j' of mode -n, landing at N - g
  constexpr int PF = 1;
  T rd[PF], rph[PF], ra[PF];
  auto column = [&](int i, bool& mir) {
    const int n = i - p.n_max;
    mir = p.sym && n < 0;
    return p.sym ? (n < 0 ? -n : n) : i;
  };
  auto load_head = [&](int i, int& jl, int& jh) {
    jl = -1; jh = -1;
    if (i >= i1) return;
    bool mir;
    const int col = column(i, mir);
    const int* jt = mir ? p.jlo_neg : p.jlo;
    const long long nj = (long long)(p.n_tiles + 1) * p.Mr;
    jl = ld<LD>(jt + bchk((long long)tile * p.Mr + col, nj, st));
    jh = ld<LD>(jt + bchk((long long)(tile + 1) * p.Mr + col, nj, st));
  };
  // A bracket table left inconsistent by a failed screen (already flagged by
  // k_bracket) must not send the reads out of [0, NRT); a window wider than
  // the tile's capacity means rays compressed beyond it (flagged here).
  auto head_ok = [&](int i, int jl, int jh) {
    if (i >= i1) return false;
    bool mir;
    column(i, mir);
    if (jl < (mir ? 2 : 1) || jh < jl || jh > p.NRT - 3) return false;
    if (jh - jl + 4 > wcap) { st |= ST_CAUSTIC; return false; }
    return true;
  };
  // ray index of window slot w (mirrored families run backwards)
  auto ray_of = [&](bool mir, int jb, int w) { return mir ? p.NRT - jb - w : jb + w; };
  auto prefetch = [&](int i, int jl, int jh) {
    bool mir;
    const int col = column(i, mir);
    const int jb = jl - 1, W = jh - jl + 4;
#pragma unroll
    for (int r = 0; r < PF; ++r) {
      const int w = lane + 32 * r;
      if (w < W) {
        const long long o = bchk((long long)ray_of(mir, jb, w) * p.Mr + col,
                                 (long long)p.NRT * p.Mr, st);
        rd[r] = ld<LD>(p.d + o);
        rph[r] = ld<LD>(p.ph + o);
        ra[r] = ld<LD>(p.a + o);
      }
    }
  };

  int i = i0 + warp;
  int jl_c, jh_c, jl_n, jh_n;
  load_head(i, jl_c, jh_c);
  load_head(i + RESUM_WARPS, jl_n, jh_n);
  bool ok_c = head_ok(i, jl_c, jh_c);
  if (ok_c) prefetch(i, jl_c, jh_c);
  for (; i < i1; i += RESUM_WARPS) {
    const bool ok = ok_c;
    const int jl = jl_c, jh = jh_c;
    bool mirrored;
    const int col = column(i, mirrored);
    const int jb = jl - 1;
    const int W = jh - jl + 4;
    const int base = mirrored ? p.N - m0 - (p.NRT - jb - p.G) * p.R : (jb - p.G) * p.R - m0;
    const T dsign = mirrored ? T(-1) : T(1);
    // FP32: the mode coefficient enters as |c_n| (scaling the amplitudes) and
    // arg(c_n) / 2 pi (added to the phases, in turns) -- cpol, formed by the
    // DFT -- so that each term is |c_n| a e^{2 pi i t}: two FMAs instead of a
    // complex product.  FP64 multiplies by c_n.
    V cn;
    T cmag = T(1), carg = T(0);
    if constexpr (sizeof(T) == 4) {
      const V cp = ld<LDC>(p.cpol + i);
      cmag = cp.x;
      carg = cp.y;
    } else {
      cn = ld<LDC>(p.c + i);
    }
    const unsigned nn = (unsigned)(i - p.n_max);
    __syncwarp();
    if (ok) {
#pragma unroll
      for (int r = 0; r < PF; ++r) {
        const int w = lane + 32 * r;
        if (w < W) {
          s_X[w] = T(base + w * p.R) + dsign * rd[r];
          if constexpr (sizeof(T) == 4) {
            s_ph[w] = rph[r] + carg;
            s_a[w] = ra[r] * cmag;
          } else {
            s_ph[w] = rph[r];
            s_a[w] = ra[r];
          }
        }
      }
      for (int w = lane + 32 * PF; w < W; w += 32) {   // beyond the prefetched rounds
        const long long o = bchk((long long)ray_of(mirrored, jb, w) * p.Mr + col,
                                 (long long)p.NRT * p.Mr, st);
        s_X[w] = T(base + w * p.R) + dsign * ld<LD>(p.d + o);
        if constexpr (sizeof(T) == 4) {
          s_ph[w] = ld<LD>(p.ph + o) + carg;
          s_a[w] = ld<LD>(p.a + o) * cmag;
        } else {
          s_ph[w] = ld<LD>(p.ph + o);
          s_a[w] = ld<LD>(p.a + o);
        }
      }
    }
    // issue the next mode's window and the following mode's brackets
    jl_c = jl_n;
    jh_c = jh_n;
    ok_c = head_ok(i + RESUM_WARPS, jl_c, jh_c);
    if (ok_c) prefetch(i + RESUM_WARPS, jl_c, jh_c);
    load_head(i + 2 * RESUM_WARPS, jl_n, jh_n);
    if (!ok) continue;
    __syncwarp();
    for (int w = 1 + lane; w <= W - 3; w += 32) {
      const T X0 = s_X[w - 1], X1 = s_X[w], X2 = s_X[w + 1], X3 = s_X[w + 2];
      const T h21 = X2 - X1, h10 = X1 - X0;
      const T r21 = T(1) / h21, r10 = T(1) / h10, r32 = T(1) / (X3 - X2);
      const T r20 = T(1) / (X2 - X0), r31 = T(1) / (X3 - X1), r30 = T(1) / (X3 - X0);
      T b0, b1, b2, b3, a0, a1, a2, a3;
      cubic_through(s_ph[w - 1], s_ph[w], s_ph[w + 1], s_ph[w + 2], r21, r10, r32, r20, r31, r30,
                    h21, h10, b0, b1, b2, b3);
      cubic_through(s_a[w - 1], s_a[w], s_a[w + 1], s_a[w + 2], r21, r10, r32, r20, r31, r30,
                    h21, h10, a0, a1, a2, a3);
      if constexpr (sizeof(T) == 4) b0 = minus_rint(b0);   // whole turns do not matter
      store_cf(s_cf + RESUM_CF * w, X1, X2, b0, b1, b2, b3, a0, a1, a2, a3);
    }
    __syncwarp();
    // Lane l sums the PW consecutive points x = l PW + q.  The interval of its
    // first point (X_w <= x < X_{w+1}, w in [1, W-3]) is guessed from the mean
    // landing spacing and corrected by comparisons; later points only step
    // forward, reloading the row when they pass X_{w+1}.
    const T xf = s_X[1];
    const T inv_sp = T(W - 3) / (s_X[W - 2] - xf);
    const int x0 = lane * PW;
    const T xv0 = T(x0);
    int w = 1 + ifloor_small(xv0 * inv_sp - xf * inv_sp);
    w = min(max(w, 1), W - 3);
    while (w > 1 && s_X[w] > xv0) --w;
    while (w < W - 3 && s_X[w + 1] <= xv0) ++w;
    T X1, X2, b0, b1, b2, b3, a0, a1, a2, a3;
    load_cf<T>(s_cf + RESUM_CF * w, X1, X2, b0, b1, b2, b3, a0, a1, a2, a3);
    if constexpr (sizeof(T) == 4) {
      // The exact integer phase n m / N mod 1 of the run's middle point,
      // moved into [-1/2, 1/2); the run's points differ from it by
      // (q - PW/2) n / N, exact in FP32 (multiples of 1/N below 2^(24 - log2 N)),
      // so each point's turn count costs one FMA.  The phase cubic is reduced
      // to (-1/2, 1/2] at its interval start, so the argument of the sine
      // stays within a few turns.
      const unsigned nmc = (nn * (unsigned)(m0 + x0 + PW / 2)) & mask;
      T bc = exact_u2f(nmc, T()) * invN;
      bc = bc >= T(0.5) ? bc - T(1) : bc;
      const T nN = T((int)nn) * invN;
#pragma unroll
      for (int q = 0; q < PW; ++q) {
        const T xv = xv0 + T(q);   // exact
        while (w < W - 3 && X2 <= xv) {
          ++w;
          load_cf<T>(s_cf + RESUM_CF * w, X1, X2, b0, b1, b2, b3, a0, a1, a2, a3);
        }
        const T tau = xv - X1;
        const T phv = ((b3 * tau + b2) * tau + b1) * tau + b0;
        const T av = ((a3 * tau + a2) * tau + a1) * tau + a0;
        const T t = fmaf(T(q - PW / 2), nN, bc) + phv;
        T sn, cs;
        sincos_turns(t, &sn, &cs);
        accr[q] = fmaf(av, cs, accr[q]);
        acci[q] = fmaf(av, sn, acci[q]);
      }
    } else {
      unsigned nm = (nn * (unsigned)(m0 + x0)) & mask;
#pragma unroll
      for (int q = 0; q < PW; ++q) {
        const T xv = xv0 + T(q);   // exact
        while (w < W - 3 && X2 <= xv) {
          ++w;
          load_cf<T>(s_cf + RESUM_CF * w, X1, X2, b0, b1, b2, b3, a0, a1, a2, a3);
        }
        const T tau = xv - X1;
        const T phv = ((b3 * tau + b2) * tau + b1) * tau + b0;
        const T av = ((a3 * tau + a2) * tau + a1) * tau + a0;
        const T t = minus_rint(exact_u2f(nm, T()) * invN + phv);
        T sn, cs;
        sincos_turns(t, &sn, &cs);
        const T ar = av * cn.x, ai = av * cn.y;
        accr[q] += ar * cs - ai * sn;
        acci[q] += ar * sn + ai * cs;
        nm = (nm + nn) & mask;
      }
    }
  }
  // fixed-order sum of the warps' partial sums
  vb_sync<BAR>(sub);
  // per warp TM points as 32 runs of PW, each run padded to PW + 1 entries so
  // that the lanes' stores fall in different banks
  V* red = reinterpret_cast<V*>(smem_raw);
  const int TMP = 32 * (PW + 1);
#pragma unroll
  for (int q = 0; q < PW; ++q) {
    V v;
    v.x = accr[q];
    v.y = acci[q];
    red[warp * TMP + lane * (PW + 1) + q] = v;
  }
  vb_sync<BAR>(sub);
  V* out = p.part + bchk((long long)group * p.N + m0, (long long)p.n_groups * p.N - (TM - 1), st);
  if (st) atomicOr(p.status, st);
  for (int x = tid; x < TM; x += RESUM_WARPS * 32) {
    const int xs = (x / PW) * (PW + 1) + x % PW;
    V sum = red[xs];
#pragma unroll
    for (int w = 1; w < RESUM_WARPS; ++w) {
      const V v = red[w * TMP + xs];
      sum.x += v.x; sum.y += v.y;
    }
    out[x] = sum;
  }
}

// FP32: 7 CTAs per SM (the register budget that keeps the one-mode-ahead
// prefetch without losing occupancy); FP64 keeps its registers
template <typename T, int PW>
__global__ void __launch_bounds__(RESUM_WARPS * 32, sizeof(T) == 4 ? 7 : 1) k_resum(const ResumArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  resum_body<T, PW, LD_NC, 0>(p, blockIdx.x, threadIdx.x, smem_raw, 0);
}

// ----------------------------------------------------------------------------
// field bookkeeping: partial sums, absorber, reflection, I/O
// ----------------------------------------------------------------------------
template <typename T, int LD>
__device__ __forceinline__ void reduce_body(const ReduceArgs<T>& p, int k) {
  using V = typename C2<T>::type;
  auto sum_at = [&](int mm) {
    V s;
    s.x = T(0); s.y = T(0);
    for (int g = 0; g < p.n_part; ++g) {
      const V v = ld<LD>(p.part + (long long)g * p.N + mm);
      s.x += v.x; s.y += v.y;
    }
    if (p.W) { const T w = p.W[mm]; s.x *= w; s.y *= w; }
    return s;
  };
  const T sg = T(p.mirror);
  if (p.sym) {
    // partials hold the physical half m in [N/2, N) and m = 0; the other
    // half is its reflection
    if (k > p.N / 2) return;
    const int m = k < p.N / 2 ? p.N / 2 + k : 0;
    const V a = sum_at(m);
    if (m == 0 || m == p.N / 2) {
      V v;
      v.x = T(0.5) * (a.x + sg * a.x); v.y = T(0.5) * (a.y + sg * a.y);
      p.u[m] = v;
    } else {
      V b;
      b.x = sg * a.x; b.y = sg * a.y;
      p.u[m] = a;
      p.u[p.N - m] = b;
    }
    return;
  }
  const int m = k;
  if (!p.mirror) {
    if (m < p.N) p.u[m] = sum_at(m);
    return;
  }
  if (m > p.N / 2) return;
  const int mm = (p.N - m) & (p.N - 1);
  const V a = sum_at(m);
  const V b = (mm == m) ? a : sum_at(mm);
  V ua, ub;
  ua.x = T(0.5) * (a.x + sg * b.x); ua.y = T(0.5) * (a.y + sg * b.y);
  ub.x = T(0.5) * (b.x + sg * a.x); ub.y = T(0.5) * (b.y + sg * a.y);
  p.u[m] = ua;
  p.u[mm] = ub;
}

template <typename T>
__global__ void k_reduce(const ReduceArgs<T> p) {
  reduce_body<T, LD_PLAIN>(p, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T>
__device__ __forceinline__ void init_body(const double* __restrict__ u0, int n_z, int N,
                                          int mirror, typename C2<T>::type* __restrict__ u,
                                          int m) {
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
__global__ void k_init(const double* __restrict__ u0, int n_z, int N, int mirror,
                       typename C2<T>::type* __restrict__ u) {
  init_body<T>(u0, n_z, N, mirror, u, blockIdx.x * blockDim.x + threadIdx.x);
}

template <typename T, int LD>
__device__ __forceinline__ void output_body(const typename C2<T>::type* __restrict__ u,
                                            int offset, int n, double* __restrict__ out, int m) {
  if (m >= n) return;
  const typename C2<T>::type v = ld<LD>(u + offset + m);
  out[2 * m] = double(v.x);
  out[2 * m + 1] = double(v.y);
}

template <typename T>
__global__ void k_output(const typename C2<T>::type* __restrict__ u, int offset, int n,
                         double* __restrict__ out) {
  output_body<T, LD_PLAIN>(u, offset, n, out, blockIdx.x * blockDim.x + threadIdx.x);
}

// ----------------------------------------------------------------------------
// (a) pruned DFT: N = N1 N2, n = n1 N2 + n2, k = k1 + N1 k2
//   X[k1 + N1 k2] = sum_n2 w_{N2}^{n2 k2} w_N^{n2 k1} sum_n1 x[n1 N2 + n2] w_{N1}^{n1 k1}
// pass 1 (N1 > 1): direct length-N1 DFTs down the columns n2, then the twiddle
// w_N^{n2 k1};
// pass 2: one CTA per kept bin n (|n| <= n_max; n >= 0 for grounded fields),
// a direct length-N2 sum along its row k1, written as c_n.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename C2<T>::type cmul(typename C2<T>::type a,
                                                     typename C2<T>::type b) {
  typename C2<T>::type r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

// pass 1: a CTA takes FFT1_COLS consecutive columns n2 (all N1 rows, one
// tile in shared memory) and forms Y[k1][n2] = w_N^{n2 k1} sum_n1 x[n1 N2 + n2]
// w_{N1}^{n1 k1} for all k1.  N1 <= 64.
// FFT1_COLS (columns per pass-1 block) is in swkb_internal.h

// (|v|, arg(v) / 2 pi) of a complex value, the angle in turns in [-1/2, 1/2].
template <typename T>
__device__ __forceinline__ typename C2<T>::type polar_turns(typename C2<T>::type v) {
  typename C2<T>::type r;
  r.x = sqrt(v.x * v.x + v.y * v.y);
  r.y = atan2(v.y, v.x) * T(0.15915494309189533577);
  return r;
}

// Field value at grid point m formed from the resummation partials: the sum
// over mode groups times the absorber, with the reflection of grounded plans
// (same arithmetic as k_reduce).
template <typename T, int LD>
__device__ __forceinline__ typename C2<T>::type field_from_parts(const FftArgs<T>& p, int m) {
  using V = typename C2<T>::type;
  const int half = p.N >> 1;
  const int src = (p.sym && m > 0 && m < half) ? p.N - m : m;
  V s;
  s.x = T(0); s.y = T(0);
  // loads issued in batches of 8, added in group order
  const V* q = p.part + src;
  int g = 0;
  for (; g + 8 <= p.n_part; g += 8) {
    V v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ld<LD>(q + (long long)(g + k) * p.N);
#pragma unroll
    for (int k = 0; k < 8; ++k) { s.x += v[k].x; s.y += v[k].y; }
  }
  for (; g < p.n_part; ++g) {
    const V v = ld<LD>(q + (long long)g * p.N);
    s.x += v.x; s.y += v.y;
  }
  if (p.W) { const T w = p.W[src]; s.x *= w; s.y *= w; }
  if (p.sym) {
    const T sg = T(p.mirror);
    if (m == 0 || m == half) {
      s.x = T(0.5) * (s.x + sg * s.x); s.y = T(0.5) * (s.y + sg * s.y);
    } else if (m < half) {
      s.x = sg * s.x; s.y = sg * s.y;
    }
  }
  return s;
}

// One pass-1 block of 256 threads (blk its index, smem_raw its shared memory).
template <typename T, int LD>
__device__ __forceinline__ void fft1_body(const FftArgs<T>& p, int blk, int tid,
                                          unsigned char* smem_raw) {
  using V = typename C2<T>::type;
  V* tile = reinterpret_cast<V*>(smem_raw);          // [N1][FFT1_COLS]
  V* w1 = tile + p.N1 * FFT1_COLS;                   // [N1] w_{N1}^k
  const int c0 = blk * FFT1_COLS;
  for (int e = tid; e < p.N1 * FFT1_COLS; e += 256) {
    const int n1 = e / FFT1_COLS, c = e % FFT1_COLS;
    const int m = n1 * p.N2 + c0 + c;
    tile[e] = p.part ? field_from_parts<T, LD>(p, m) : ld<LD>(p.u + m);
  }
  for (int k = tid; k < p.N1; k += 256) w1[k] = p.tw[(long long)k * p.N2];
  __syncthreads();
  for (int e = tid; e < p.N1 * FFT1_COLS; e += 256) {
    const int k1 = e / FFT1_COLS, c = e % FFT1_COLS;
    V acc;
    acc.x = T(0); acc.y = T(0);
    for (int n1 = 0; n1 < p.N1; ++n1) {
      const V t = cmul<T>(tile[n1 * FFT1_COLS + c], w1[(n1 * k1) & (p.N1 - 1)]);
      acc.x += t.x; acc.y += t.y;
    }
    const int n2 = c0 + c;
    p.Y[(long long)k1 * p.N2 + n2] = cmul<T>(acc, p.tw[(long long)n2 * k1]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fft1(const FftArgs<T> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fft1_body<T, LD_PLAIN>(p, blockIdx.x, threadIdx.x, smem_raw);
}

// out_i = c_i f_i (mode coefficients of a plane between screens), and its
// polar form when pol is given.
template <typename T>
__global__ void k_cscale(const typename C2<T>::type* __restrict__ c,
                         const typename C2<T>::type* __restrict__ f,
                         typename C2<T>::type* __restrict__ out,
                         typename C2<T>::type* __restrict__ pol, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const typename C2<T>::type v = cmul<T>(c[i], f[i]);
  out[i] = v;
  if (pol) pol[i] = polar_turns<T>(v);
}

// w_{N2}^{idx} from the table of w_N (w_{N2} = w_N^{N1}).
template <typename V>
__device__ __forceinline__ V twiddle2(const V* tw, unsigned idx, int, int N1) {
  return tw[(long long)idx * N1];
}

// pass 2: one CTA (4 warps) per kept mode n:
// X[k1 + N1 k2] = sum_n2 Y[k1][n2] w_{N2}^{n2 k2} (direct, pruned: only the
// 2 n_max + 1 kept bins are formed); c_n = X / N times the range-phase carry.
constexpr int FFT2_THREADS = 128;

// One pass-2 block of FFT2_THREADS threads: blk its index (one kept mode),
// wsum FFT2_THREADS / 32 values of shared memory, sub the barrier slot (BAR).
template <typename T, int LD, int BAR>
__device__ __forceinline__ void fft2_body(const FftArgs<T>& p, int blk, int tid,
                                          typename C2<T>::type* wsum, int sub) {
  using V = typename C2<T>::type;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  // grounded fields are even / odd, so c_{-n} = +-c_n: only n >= 0 is formed
  const int i = blk + (p.mirror ? p.n_max : 0);
  const int n = i - p.n_max;
  const int b = n >= 0 ? n : n + p.N;
  const int k1 = b & (p.N1 - 1);
  const int k2 = b / p.N1;
  const V* row = (p.N1 > 1 ? p.Y : p.u) + (long long)k1 * p.N2;
  V acc;
  acc.x = T(0); acc.y = T(0);
  // row entries and twiddles loaded 8 iterations at a time, summed in order
  constexpr int B = 8;
  int n2 = tid;
  for (; n2 + (B - 1) * FFT2_THREADS < p.N2; n2 += B * FFT2_THREADS) {
    V rv[B], tv[B];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int m = n2 + k * FFT2_THREADS;
      const unsigned e = (unsigned)(((long long)m * k2) & (p.N2 - 1));
      rv[k] = ld<LD>(row + m);
      tv[k] = twiddle2(p.tw, e, p.log2N2, p.N1);
    }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const V t = cmul<T>(rv[k], tv[k]);
      acc.x += t.x; acc.y += t.y;
    }
  }
  for (; n2 < p.N2; n2 += FFT2_THREADS) {
    const unsigned e = (unsigned)(((long long)n2 * k2) & (p.N2 - 1));
    const V t = cmul<T>(ld<LD>(row + n2), twiddle2(p.tw, e, p.log2N2, p.N1));
    acc.x += t.x; acc.y += t.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if (lane == 0) wsum[warp] = acc;
  vb_sync<BAR>(sub);
  if (tid == 0) {
    V tot = wsum[0];
#pragma unroll
    for (int w = 1; w < FFT2_THREADS / 32; ++w) { tot.x += wsum[w].x; tot.y += wsum[w].y; }
    tot.x *= p.inv_N; tot.y *= p.inv_N;
    const V cv = cmul<T>(tot, p.ephi[i]);
    p.c[i] = cv;
    if (p.mirror && n > 0) {
      V cm;
      cm.x = T(p.mirror) * cv.x; cm.y = T(p.mirror) * cv.y;
      p.c[2 * p.n_max - i] = cm;
    }
    if (p.cpol) {   // |c_n| and arg(c_n) / 2 pi (turns, in (-1/2, 1/2])
      V pol = polar_turns<T>(cv);
      p.cpol[i] = pol;
      if (p.mirror && n > 0) {
        if (p.mirror < 0) pol.y = pol.y > T(0) ? pol.y - T(0.5) : pol.y + T(0.5);
        p.cpol[2 * p.n_max - i] = pol;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(FFT2_THREADS) k_fft2(const FftArgs<T> p) {
  __shared__ typename C2<T>::type wsum[FFT2_THREADS / 32];
  fft2_body<T, LD_PLAIN, 0>(p, blockIdx.x, threadIdx.x, wsum, 0);
}

}  // namespace swkb
