// Separation-of-variables reference on the GPU (Sec. 3.1, Eqs. series_sol,
// phi_equation, series_init, sl_expansion), all in FP64:
//
//   1. eh_j, the period means of eps cos(kappa_j s), j = 0..2K, from n_q + 1
//      samples on the half period (type-1 cosine sums, exact integer phase
//      index (j i) mod 2 n_q);
//   2. the Galerkin matrices of phi'' + k^2 eps phi in the cosine and sine
//      bases about the symmetry point (real symmetric, K + 1 and K rows,
//      padded to an even size P with zero rows);
//   3. their eigenpairs by parallel cyclic Jacobi: each sweep runs the P - 1
//      rounds of a round-robin tournament, a round rotating the P / 2
//      disjoint index pairs (p, q) at once in one kernel (a thread per 2 x 2
//      block of the upper triangle, folded so that no lane idles), which
//      also makes the next round's rotations; one sweep is one CUDA graph,
//      replayed until the off-diagonal norm falls below 1e-15 of the
//      Frobenius norm.  The eigenvalues are the diagonal; the eigenvectors
//      stay implicit: the field's basis projections are rotated along
//      (a = W uh) and the rotations are logged, so that W^T is applied to the
//      advanced coefficients by replaying the log backwards;
//   4. the projections of the field on the basis (period means), the
//      advance by exp(i alpha x) and the sum back onto the field points.
//
// FP64 throughput is the scarce resource on this GPU (two FMAs per SM and
// clock), so the rotation tangent is found in FP32 and only c, s and the
// updates are FP64.  A zero padding row never mixes with the others (its
// off-diagonal entries stay exactly zero, so its rotations are the
// identity), and every block and its transpose are written from one
// computation, so A stays exactly symmetric.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "swkb.h"
#include "swkb_internal.h"

namespace {

swkb_status hfail(swkb_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  swkb::set_last_error(buf);
  return s;
}

#define HCK(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return hfail(e_ == cudaErrorMemoryAllocation ? SWKB_ERR_OOM : SWKB_ERR_CUDA,          \
                   "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,        \
                   __LINE__);                                                               \
  } while (0)

#define HTRY(expr)                    \
  do {                                \
    swkb_status s_ = (expr);          \
    if (s_ != SWKB_OK) return s_;     \
  } while (0)

constexpr int kMaxSweeps = 60;
constexpr double kTol = 1e-15;
constexpr int kThreads = 256;
// Jacobi rounds use small CTAs: a round has only P^2 / 8 blocks of work, and
// spreading them evenly over the SMs matters more than CTA size
constexpr int kRoundThreads = 64;

// round r (0 <= r < P - 1) of the circle tournament on P players: pair i
// is (P - 1, r) for i = 0 and ((r + i) mod m, (r - i) mod m), m = P - 1,
// otherwise (0 <= r, i < m, so one conditional add or subtract reduces)
__host__ __device__ inline void rr_pair(int r, int i, int P, int& p, int& q) {
  const int m = P - 1;
  if (i == 0) {
    p = m;
    q = r;
  } else {
    p = r + i;
    if (p >= m) p -= m;
    q = r - i;
    if (q < 0) q += m;
  }
}

int grid_for(long long work, int threads = kThreads) {
  const long long b = (work + threads - 1) / threads;
  return (int)std::min<long long>(std::max<long long>(b, 1), 152LL * 64);
}

// ---------------------------------------------------------------------------
// tables and the Galerkin matrices
// ---------------------------------------------------------------------------

// tab[r] = (cos, sin)(2 pi r / N)
__global__ void k_period_table(double2* tab, int N) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)r / (double)N, &s, &c);
    tab[r] = make_double2(c, s);
  }
}

// tq[r] = cos(pi r / n_q), r < 2 n_q
__global__ void k_dct_table(double* tq, int n_q) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < 2LL * n_q;
       r += (long long)gridDim.x * blockDim.x)
    tq[r] = cospi((double)r / (double)n_q);
}

__device__ inline double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;   // valid in thread 0
}

// eh[b][j] = (1 / 2 n_q) [e_0 + 2 sum_{0<i<n_q} e_i cos(pi j i / n_q) + e_{n_q} cos(pi j)]
// one CTA per (j, b)
__global__ void k_eps_means(const double* eps, int n_q, const double* tq, int J, double* eh) {
  __shared__ double sh[32];
  const int j = blockIdx.x, b = blockIdx.y;
  const double* e = eps + (size_t)b * (n_q + 1);
  const long long two = 2LL * n_q;
  double acc = 0.0;
  for (int i = 1 + threadIdx.x; i < n_q; i += blockDim.x)
    acc += e[i] * tq[((long long)j * i) % two];
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0)
    eh[(size_t)b * J + j] = (e[0] + 2.0 * acc + ((j & 1) ? -e[n_q] : e[n_q])) / (double)two;
}

struct HillDims {
  int K, P, n_par, par0;   // par0: parity of the first block (0 cosines, 1 sines)
  double kappa1;           // 2 pi / L
};

__device__ inline int parity_of(const HillDims& d, int mat) {
  return d.n_par == 2 ? (mat & 1) : d.par0;
}

// A[mat] and W[mat] = I; mat = b n_par + block
__global__ void k_build(HillDims d, int n_mat, const double* k, const double* eh, double* A,
                        double* W) {
  const long long PP = (long long)d.P * d.P, total = PP * n_mat;
  const int J = 2 * d.K + 1;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mat = (int)(idx / PP);
    const int rem = (int)(idx - (long long)mat * PP);
    const int r = rem / d.P, c = rem - r * d.P;
    const int odd = parity_of(d, mat);
    const int n_blk = odd ? d.K : d.K + 1;
    double a = 0.0;
    if (r < n_blk && c < n_blk) {
      const int b = mat / d.n_par;
      const int bn = r + odd, bm = c + odd;   // basis indices
      const double* e = eh + (size_t)b * J;
      const double wn = bn == 0 ? 1.0 : M_SQRT2, wm = bm == 0 ? 1.0 : M_SQRT2;
      const double sum = e[abs(bn - bm)] + (odd ? -e[bn + bm] : e[bn + bm]);
      a = k[b] * k[b] * (wn * wm) * sum * 0.5;
      if (r == c) {
        const double kap = d.kappa1 * bn;
        a -= kap * kap;
      }
    }
    A[idx] = a;
    if (W) W[idx] = r == c ? 1.0 : 0.0;
  }
}

// symmetric part of a caller matrix, padded to P
__global__ void k_load_sym(const double* in, int n, int P, int n_mat, double* A, double* W) {
  const long long PP = (long long)P * P, total = PP * n_mat;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mat = (int)(idx / PP);
    const int rem = (int)(idx - (long long)mat * PP);
    const int r = rem / P, c = rem - r * P;
    double a = 0.0;
    if (r < n && c < n) {
      const double* m = in + (size_t)mat * n * n;
      a = 0.5 * (m[(size_t)r * n + c] + m[(size_t)c * n + r]);
    }
    A[idx] = a;
    if (W) W[idx] = r == c ? 1.0 : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Jacobi rounds
// ---------------------------------------------------------------------------

// The rotation (c, s) of a pair: t = tan(theta) is the root of
// t^2 + 2 t th - 1 = 0 of smaller magnitude, th = (a_qq - a_pp) / (2 a_pq),
// found in FP32 (FP64 instructions are scarce here), then c = 1 / sqrt(1 +
// t^2) and s = t c in FP64, so that J stays orthogonal to FP64 rounding: an
// FP32 tangent leaves |a'_pq| ~ 1e-7 |a_pq|, which the following sweeps
// remove like any other off-diagonal entry.  Operands FP32 cannot hold take
// the FP64 formula.
__device__ inline double2 rotation(double app, double aqq, double apq) {
  if (apq == 0.0) return make_double2(1.0, 0.0);
  const double d = aqq - app;
  double t;
  if (fabs(apq) > 1e-30 && fabs(apq) < 1e30 && fabs(d) < 1e30) {
    const float th = (float)d / (2.0f * (float)apq);
    const float ath = fabsf(th);
    t = ath > 1e18f ? 0.5f / th : copysignf(1.0f, th) / (ath + sqrtf(1.0f + th * th));
  } else {
    const double th = d / (2.0 * apq);
    const double ath = fabs(th);
    t = ath > 1e150 ? 0.5 / th : copysign(1.0, th) / (ath + sqrt(1.0 + th * th));
  }
  const double c = rsqrt(1.0 + t * t);
  return make_double2(c, t * c);
}

// player a in round r: its pair, whether it is the pair's p, and its partner
// (the pairs i >= 1 of a round have p + q = 2 r mod m)
__device__ inline int player_pair(int a, int r, int P, bool& is_p, int& partner) {
  const int m = P - 1, npair = P / 2;
  if (a == m) {
    is_p = true;
    partner = r;
    return 0;
  }
  if (a == r) {
    is_p = false;
    partner = m;
    return 0;
  }
  int d = a - r;
  if (d < 0) d += m;
  if (d < npair) {
    is_p = true;
    partner = r - d;
    if (partner < 0) partner += m;
    return d;
  }
  is_p = false;
  partner = r + (m - d);
  if (partner >= m) partner -= m;
  return m - d;
}

// rotations of one round from A (the first round of the first sweep)
__global__ void k_rotations(const double* __restrict__ A, int P, int n_mat, int round,
                            double2* __restrict__ rot) {
  const int npair = P / 2;
  const long long total = (long long)n_mat * npair;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mat = (int)(idx / npair), i = (int)(idx - (long long)mat * npair);
    int p, q;
    rr_pair(round, i, P, p, q);
    const double* a = A + (size_t)mat * P * P;
    rot[idx] = rotation(a[(size_t)p * P + p], a[(size_t)q * P + q], a[(size_t)p * P + q]);
  }
}

// R = J_u^T B J_v with J = [[c, s], [-s, c]] on (p, q)
__device__ inline void rotate_block(double cu, double su, double cv, double sv, double b00,
                                    double b01, double b10, double b11, double& r00,
                                    double& r01, double& r10, double& r11) {
  const double l00 = cu * b00 - su * b10, l01 = cu * b01 - su * b11;
  const double l10 = su * b00 + cu * b10, l11 = su * b01 + cu * b11;
  r00 = l00 * cv - l01 * sv;
  r01 = l00 * sv + l01 * cv;
  r10 = l10 * cv - l11 * sv;
  r11 = l10 * sv + l11 * cv;
}

// One round: A <- J^T A J, a thread per 2 x 2 block (i <= j, which also
// writes the transposed block (j, i); the upper triangle of blocks is folded
// into a rectangle so no lane idles); with WITH_W, W <- J^T W, a thread per
// column and pair; with vec, v <- J^T v for one complex vector per matrix, a
// thread per pair.  The rotations of the next round are made here too:
// their operands a_pp, a_qq, a_pq are written by three threads of this
// round, each of which, after its writes and a fence, counts itself in on
// the pair's counter; the third computes the rotation (reading the operands
// from L2) and resets the counter.  No thread waits on another.
//
// Operands are read through L2 (ld.global.cg): they were written by other
// CTAs, in this round's predecessor or, for the next rotations, in this one.
template <bool WITH_W>
__device__ __forceinline__ void round_items(double* __restrict__ A, double* __restrict__ W,
                                            double2* __restrict__ vec, int P, int n_mat,
                                            int round, const double2* __restrict__ rot,
                                            double2* __restrict__ rot_next,
                                            unsigned* __restrict__ cnt, long long first,
                                            long long stride) {
  const int npair = P / 2;
  const int next = round + 1 == P - 1 ? 0 : round + 1;
  const long long nb = (long long)((npair + 1) / 2) * (npair + 1);
  const long long nw = WITH_W ? (long long)npair * P : 0;
  const long long nv = vec ? npair : 0;
  const long long per = nb + nw + nv, total = per * n_mat;
  for (long long idx = first; idx < total; idx += stride) {
    const int mat = (int)(idx / per);
    long long rem = idx - (long long)mat * per;
    double* a = A + (size_t)mat * P * P;
    const double2* rm = rot + (size_t)mat * npair;
    if (rem < nb) {
      const int rr = (int)(rem / (npair + 1)), cc = (int)(rem - (long long)rr * (npair + 1));
      int i, j;
      if (cc < npair - rr) {
        i = rr;
        j = rr + cc;
      } else {
        i = npair - 1 - rr;
        if (i == rr) continue;   // the middle row of an odd count is done once
        j = i + (cc - (npair - rr));
      }
      int pi, qi, pj, qj;
      rr_pair(round, i, P, pi, qi);
      rr_pair(round, j, P, pj, qj);
      const double2 ri = __ldcg(rm + i), rj = __ldcg(rm + j);
      double* e00 = a + (size_t)pi * P + pj;
      double* e01 = a + (size_t)pi * P + qj;
      double* e10 = a + (size_t)qi * P + pj;
      double* e11 = a + (size_t)qi * P + qj;
      if (i == j) {
        // the pair's own block in a form without cancellation at the scale
        // of a_pp (exact for any rotation, not only the annihilating one):
        // delta = s (2 c a_pq - s d), d = a_qq - a_pp; a'_pp = a_pp - delta,
        // a'_qq = a_qq + delta, a'_pq = (c - s)(c + s) a_pq - c s d
        const double c = ri.x, sn = ri.y;
        const double app = __ldcg(e00), aqq = __ldcg(e11), apq = __ldcg(e01), d = aqq - app;
        const double delta = sn * (2.0 * c * apq - sn * d);
        const double off = (c - sn) * (c + sn) * apq - c * sn * d;
        *e00 = app - delta;
        *e11 = aqq + delta;
        *e01 = off;
        *e10 = off;
      } else {
        double r00, r01, r10, r11;
        rotate_block(ri.x, ri.y, rj.x, rj.y, __ldcg(e00), __ldcg(e01), __ldcg(e10), __ldcg(e11),
                     r00, r01, r10, r11);
        *e00 = r00;
        *e01 = r01;
        *e10 = r10;
        *e11 = r11;
        a[(size_t)pj * P + pi] = r00;
        a[(size_t)qj * P + pi] = r01;
        a[(size_t)pj * P + qi] = r10;
        a[(size_t)qj * P + qi] = r11;
      }
      // The next round's operands among the entries written here.  Rows pi
      // and qi each have one partner next round; where it is a column of
      // this block, the block holds that pair's a_pq (once: (p, q) and
      // (q, p) are written together).  A diagonal block also holds a_pp of
      // its two rows' pairs, and, for P = 2 only (one round per sweep), the
      // same pair's a_pq.
      bool is_p;
      int tp, tq;
      const int kp = player_pair(pi, next, P, is_p, tp);
      const int kq = player_pair(qi, next, P, is_p, tq);
      int key0 = -1, key1 = -1, key2 = -1;
      if (i == j) {
        key0 = kp;
        key1 = kq;
        if (tp == qi) key2 = kp;
      } else {
        if (tp == pj || tp == qj) key0 = kp;
        if (tq == pj || tq == qj) {
          if (key0 < 0) key0 = kq;
          else key1 = kq;
        }
      }
      if (key0 < 0) continue;
      __threadfence();
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const int key = e == 0 ? key0 : (e == 1 ? key1 : key2);
        if (key < 0) break;
        unsigned* c = cnt + (size_t)mat * npair + key;
        if (atomicAdd(c, 1u) == 2u) {
          __threadfence();
          int p, q;
          rr_pair(next, key, P, p, q);
          rot_next[(size_t)mat * npair + key] =
              rotation(__ldcg(a + (size_t)p * P + p), __ldcg(a + (size_t)q * P + q),
                       __ldcg(a + (size_t)p * P + q));
          *c = 0u;
        }
      }
    } else if (WITH_W && rem < nb + nw) {
      rem -= nb;
      const int i = (int)(rem / P), col = (int)(rem - (long long)i * P);
      int p, q;
      rr_pair(round, i, P, p, q);
      double* w = W + (size_t)mat * P * P;
      const double2 r = __ldcg(rm + i);
      const double wp = __ldcg(w + (size_t)p * P + col), wq = __ldcg(w + (size_t)q * P + col);
      w[(size_t)p * P + col] = r.x * wp - r.y * wq;
      w[(size_t)q * P + col] = r.y * wp + r.x * wq;
    } else {
      const int i = (int)(rem - nb - nw);
      int p, q;
      rr_pair(round, i, P, p, q);
      double2* v = vec + (size_t)mat * P;
      const double2 r = __ldcg(rm + i);
      const double2 vp = __ldcg(v + p), vq = __ldcg(v + q);
      v[p] = make_double2(r.x * vp.x - r.y * vq.x, r.x * vp.y - r.y * vq.y);
      v[q] = make_double2(r.y * vp.x + r.x * vq.x, r.y * vp.y + r.x * vq.y);
    }
  }
}

// one round per launch
template <bool WITH_W>
__global__ void k_round(double* __restrict__ A, double* __restrict__ W,
                        double2* __restrict__ vec, int P, int n_mat, int round,
                        const double2* __restrict__ rot, double2* __restrict__ rot_next,
                        unsigned* __restrict__ cnt) {
  round_items<WITH_W>(A, W, vec, P, n_mat, round, rot, rot_next, cnt,
                      blockIdx.x * (long long)blockDim.x + threadIdx.x,
                      (long long)gridDim.x * blockDim.x);
}

// Replays the logged rotations backwards on complex vectors, v <- J v from
// the last round to the first (v <- W^T v), one CTA per vector held in
// shared memory.  Each thread fetches its next round's rotations before the
// current round's barrier.
constexpr int kReplayMaxPerThread = 4;

__global__ void k_replay(const double2* __restrict__ log, int n_rounds, int P, int n_mat,
                         int vecs_per_mat, double2* __restrict__ vecs) {
  extern __shared__ double2 v[];
  const int npair = P / 2;
  const int vec = blockIdx.x, mat = vec / vecs_per_mat;
  double2* gv = vecs + (size_t)vec * P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) v[i] = gv[i];
  auto rot_at = [&](int step, int i) {
    return log[((size_t)(n_rounds - 1 - step) * n_mat + mat) * npair + i];
  };
  double2 cur[kReplayMaxPerThread];
  for (int k = 0; k < kReplayMaxPerThread; ++k) {
    const int i = threadIdx.x + k * blockDim.x;
    if (i < npair && n_rounds > 0) cur[k] = rot_at(0, i);
  }
  __syncthreads();
  for (int step = 0; step < n_rounds; ++step) {
    const int r = (n_rounds - 1 - step) % (P - 1);
    double2 nxt[kReplayMaxPerThread];
    for (int k = 0; k < kReplayMaxPerThread; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i < npair && step + 1 < n_rounds) nxt[k] = rot_at(step + 1, i);
    }
    for (int k = 0; k < kReplayMaxPerThread; ++k) {
      const int i = threadIdx.x + k * blockDim.x;
      if (i >= npair) break;
      int p, q;
      rr_pair(r, i, P, p, q);
      const double c = cur[k].x, s = cur[k].y;
      const double2 vp = v[p], vq = v[q];
      v[p] = make_double2(c * vp.x + s * vq.x, c * vp.y + s * vq.y);
      v[q] = make_double2(c * vq.x - s * vp.x, c * vq.y - s * vp.y);
    }
    for (int k = 0; k < kReplayMaxPerThread; ++k) cur[k] = nxt[k];
    __syncthreads();
  }
  for (int i = threadIdx.x; i < P; i += blockDim.x) gv[i] = v[i];
}

// norms[mat] = (sum of squared off-diagonal entries, sum of all squares)
__global__ void k_norms(const double* A, int P, double* norms) {
  __shared__ double sh[32];
  const int mat = blockIdx.y;
  const double* a = A + (size_t)mat * P * P;
  const long long PP = (long long)P * P;
  double off = 0.0, all = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < PP;
       idx += (long long)gridDim.x * blockDim.x) {
    const double v = a[idx];
    const long long r = idx / P;
    all += v * v;
    if (idx != r * P + r) off += v * v;
  }
  off = block_sum(off, sh);
  __syncthreads();
  all = block_sum(all, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&norms[2 * mat], off);
    atomicAdd(&norms[2 * mat + 1], all);
  }
}

// ---------------------------------------------------------------------------
// projection, advance, synthesis
// ---------------------------------------------------------------------------

struct FieldDims {
  int n_z, N, m_c, mirror;   // mirror: 0 periodic, +1 Neumann, -1 Dirichlet
};

// the field at period point i (the S-WKB mirror for grounded domains)
__device__ inline double2 field_at(const double2* u, const FieldDims& f, int i) {
  if (f.mirror == 0) return u[i];
  if (i >= f.n_z) return u[i - f.n_z];
  if (i == 0) return make_double2(0.0, 0.0);
  const double2 v = u[f.n_z - i];
  return f.mirror > 0 ? v : make_double2(-v.x, -v.y);
}

// uh[mat][row] = w_n / N sum_i u(i) e_n(i); one CTA per (row, mat)
__global__ void k_project(const double2* u0, FieldDims f, HillDims d, const double2* tab,
                          double2* uh) {
  __shared__ double sh[32];
  const int row = blockIdx.x, mat = blockIdx.y;
  const int odd = parity_of(d, mat);
  const int n_blk = odd ? d.K : d.K + 1;
  const int b = mat / d.n_par;
  double sr = 0.0, si = 0.0;
  if (row < n_blk) {
    const int bn = row + odd;
    const double2* u = u0 + (size_t)b * f.n_z;
    for (int i = threadIdx.x; i < f.N; i += blockDim.x) {
      long long ph = ((long long)bn * (i - f.m_c)) % f.N;
      if (ph < 0) ph += f.N;
      const double2 cs = tab[ph];
      const double e = odd ? cs.y : cs.x;
      const double2 v = field_at(u, f, i);
      sr += v.x * e;
      si += v.y * e;
    }
  }
  sr = block_sum(sr, sh);
  __syncthreads();
  si = block_sum(si, sh);
  if (threadIdx.x == 0) {
    const double w = (row < n_blk && row + odd > 0) ? M_SQRT2 : 1.0;
    const double sc = row < n_blk ? w / (double)f.N : 0.0;
    uh[(size_t)mat * d.P + row] = make_double2(sr * sc, si * sc);
  }
}

// ph[mat][r][j] = a_j exp(i alpha_j x_r), alpha_j = sqrt(lambda_j) (principal)
__global__ void k_advance_coefficients(const double* A, const double2* coef, HillDims d,
                                       int n_mat, const double* xs, int n_x, double2* ph) {
  const long long total = (long long)n_mat * n_x * d.P;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % d.P);
    const long long mr = idx / d.P;
    const int r = (int)(mr % n_x), mat = (int)(mr / n_x);
    const int n_blk = parity_of(d, mat) ? d.K : d.K + 1;
    double2 out = make_double2(0.0, 0.0);
    if (j < n_blk) {
      const double lam = A[(size_t)mat * d.P * d.P + (size_t)j * d.P + j];
      const double2 a = coef[(size_t)mat * d.P + j];
      const double x = xs[r];
      double er, ei;
      if (lam >= 0.0) {
        double s, c;
        sincos(sqrt(lam) * x, &s, &c);
        er = c;
        ei = s;
      } else {
        er = exp(-sqrt(-lam) * x);
        ei = 0.0;
      }
      out = make_double2(a.x * er - a.y * ei, a.x * ei + a.y * er);
    }
    ph[idx] = out;
  }
}

// u_out[b][r][m] = sum over blocks and rows of g e_n at the field point m
__global__ void k_synthesize(const double2* g, FieldDims f, HillDims d, int batch, int n_x,
                             const double2* tab, double2* out) {
  const long long total = (long long)batch * n_x * f.n_z;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(idx % f.n_z);
    const long long br = idx / f.n_z;
    const int r = (int)(br % n_x), b = (int)(br / n_x);
    const int i = f.mirror ? f.n_z + m : m;   // period point
    double sr = 0.0, si = 0.0;
    for (int blk = 0; blk < d.n_par; ++blk) {
      const int mat = b * d.n_par + blk;
      const int odd = parity_of(d, mat);
      const int n_blk = odd ? d.K : d.K + 1;
      const double2* gg = g + ((size_t)mat * n_x + r) * d.P;
      for (int row = 0; row < n_blk; ++row) {
        const int bn = row + odd;
        long long ph = ((long long)bn * (i - f.m_c)) % f.N;
        if (ph < 0) ph += f.N;
        const double2 cs = tab[ph];
        const double e = (bn == 0 ? 1.0 : M_SQRT2) * (odd ? cs.y : cs.x);
        sr += gg[row].x * e;
        si += gg[row].y * e;
      }
    }
    out[idx] = make_double2(sr, si);
  }
}

// eigenvalues of the real rows: lam[b][offset of block + j]
__global__ void k_eigenvalues(const double* A, HillDims d, int batch, double* lam) {
  const int n_eig = d.n_par == 2 ? 2 * d.K + 1 : (d.par0 ? d.K : d.K + 1);
  const long long total = (long long)batch * n_eig;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(idx / n_eig), e = (int)(idx - (long long)b * n_eig);
    int blk = 0, j = e;
    if (d.n_par == 2 && e > d.K) {
      blk = 1;
      j = e - (d.K + 1);
    }
    const int mat = b * d.n_par + blk;
    lam[idx] = A[(size_t)mat * d.P * d.P + (size_t)j * d.P + j];
  }
}

__global__ void k_copy_leading(const double* A, const double* W, int n, int P, int n_mat,
                               double* lam, double* vec) {
  const long long nn = (long long)n * n, total = nn * n_mat;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int mat = (int)(idx / nn);
    const long long rem = idx - (long long)mat * nn;
    const int r = (int)(rem / n), c = (int)(rem - (long long)r * n);
    const size_t src = (size_t)mat * P * P + (size_t)r * P + c;
    if (vec) vec[idx] = W[src];
    if (lam && r == c) lam[(size_t)mat * n + r] = A[src];
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// device buffers of one call, released on every exit path
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t sweep = nullptr;
  double* host_norms = nullptr;
  ~Scratch() {
    if (stream) cudaStreamSynchronize(stream);
    if (sweep) cudaGraphExecDestroy(sweep);
    for (void* p : ptrs) cudaFree(p);
    if (host_norms) cudaFreeHost(host_norms);
    if (stream) cudaStreamDestroy(stream);
  }
  template <typename T>
  swkb_status alloc(T** p, size_t count) {
    void* v = nullptr;
    HCK(cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T)));
    ptrs.push_back(v);
    *p = (T*)v;
    return SWKB_OK;
  }
  // frees one buffer now, after the stream's work on it
  swkb_status release(void* p) {
    HCK(cudaStreamSynchronize(stream));
    for (size_t i = 0; i < ptrs.size(); ++i)
      if (ptrs[i] == p) {
        ptrs.erase(ptrs.begin() + i);
        HCK(cudaFree(p));
        break;
      }
    return SWKB_OK;
  }
};

// Rotations of every round of every sweep, in order, (c, s) per pair:
// log[(round * n_mat + mat) * P / 2 + pair]
struct RotLog {
  double2* d = nullptr;
  int rounds = 0;
};

// Jacobi sweeps on A (n_mat matrices of P x P; W and vec, one complex
// vector per matrix, rotated along when not NULL) until converged.  A sweep (P - 1 fused rounds and the norms) is captured once as
// a graph; rotations live in P slots of a round each: round r reads slot r
// and makes the next round's in slot r + 1, the last round the next sweep's
// first in slot P - 1, which the sweep's first node copies to slot 0.  With
// log, slots 0..P-2 are appended to it after every sweep.
swkb_status jacobi(Scratch& s, double* A, double* W, double2* vec, int P, int n_mat,
                   int* sweeps_out, RotLog* log) {
  const int npair = P / 2;
  const size_t per_round = (size_t)n_mat * npair;
  double2* slots = nullptr;
  unsigned* cnt = nullptr;
  double* norms = nullptr;
  HTRY(s.alloc(&slots, (size_t)P * per_round));
  HTRY(s.alloc(&cnt, per_round));
  HTRY(s.alloc(&norms, 2 * (size_t)n_mat));
  HCK(cudaMallocHost(&s.host_norms, 2 * sizeof(double) * n_mat));
  HCK(cudaMemsetAsync(cnt, 0, per_round * sizeof(unsigned), s.stream));
  const long long work = (long long)n_mat * ((long long)((npair + 1) / 2) * (npair + 1) +
                                             (W ? (long long)npair * P : 0) + (vec ? npair : 0));
  const int g_round = grid_for(work, kRoundThreads);
  const int norm_cols = std::max(1, std::min(64, (int)(((long long)P * P + 4095) / 4096)));
  double2* last = slots + (size_t)(P - 1) * per_round;
  cudaGraph_t graph = nullptr;
  HCK(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
  cudaMemcpyAsync(slots, last, per_round * sizeof(double2), cudaMemcpyDeviceToDevice, s.stream);
  for (int r = 0; r < P - 1; ++r) {
    const double2* cur = slots + (size_t)r * per_round;
    double2* nxt = slots + (size_t)(r + 1) * per_round;   // slot P - 1 after the last round
    if (W)
      k_round<true><<<g_round, kRoundThreads, 0, s.stream>>>(A, W, vec, P, n_mat, r, cur, nxt,
                                                              cnt);
    else
      k_round<false><<<g_round, kRoundThreads, 0, s.stream>>>(A, nullptr, vec, P, n_mat, r, cur,
                                                               nxt, cnt);
  }
  cudaMemsetAsync(norms, 0, 2 * sizeof(double) * n_mat, s.stream);
  k_norms<<<dim3(norm_cols, n_mat), kThreads, 0, s.stream>>>(A, P, norms);
  cudaMemcpyAsync(s.host_norms, norms, 2 * sizeof(double) * n_mat, cudaMemcpyDeviceToHost,
                  s.stream);
  const cudaError_t ec = cudaStreamEndCapture(s.stream, &graph);
  if (ec != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return hfail(SWKB_ERR_CUDA, "sweep capture failed: %s", cudaGetErrorString(ec));
  }
  const cudaError_t ei = cudaGraphInstantiate(&s.sweep, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return hfail(SWKB_ERR_CUDA, "sweep graph: %s", cudaGetErrorString(ei));
  // the Frobenius norms are invariant under the rotations: take them before;
  // the first round's rotations go to slot P - 1
  HCK(cudaMemsetAsync(norms, 0, 2 * sizeof(double) * n_mat, s.stream));
  k_norms<<<dim3(norm_cols, n_mat), kThreads, 0, s.stream>>>(A, P, norms);
  k_rotations<<<grid_for((long long)per_round), kThreads, 0, s.stream>>>(A, P, n_mat, 0, last);
  HCK(cudaGetLastError());
  HCK(cudaMemcpyAsync(s.host_norms, norms, 2 * sizeof(double) * n_mat, cudaMemcpyDeviceToHost,
                      s.stream));
  HCK(cudaStreamSynchronize(s.stream));
  std::vector<double> fro(n_mat);
  for (int m = 0; m < n_mat; ++m) {
    fro[m] = s.host_norms[2 * m + 1];
    if (!std::isfinite(fro[m]))
      return hfail(SWKB_ERR_INVALID_ARG, "matrix %d has non-finite entries", m);
  }
  const size_t sweep_log = (size_t)(P - 1) * per_round;
  // SWKB_HILL_LOG_SWEEPS: the log's first capacity in sweeps (tests set it
  // to 1 to exercise its growth)
  const char* lc = getenv("SWKB_HILL_LOG_SWEEPS");
  const int first_cap = lc ? std::max(1, atoi(lc)) : 8;
  double2* logbuf = nullptr;
  int log_cap = 0;
  int sweeps = 0;
  bool done = true;
  for (int m = 0; m < n_mat; ++m) done = done && s.host_norms[2 * m] <= kTol * kTol * fro[m];
  while (!done) {
    if (sweeps == kMaxSweeps)
      return hfail(SWKB_ERR_INVALID_ARG, "Jacobi iteration did not converge in %d sweeps",
                   kMaxSweeps);
    HCK(cudaGraphLaunch(s.sweep, s.stream));
    if (log) {
      if (sweeps == log_cap) {   // room for twice as many sweeps (8 at first)
        const int cap = log_cap ? 2 * log_cap : first_cap;
        double2* grown = nullptr;
        HTRY(s.alloc(&grown, (size_t)cap * sweep_log));
        if (logbuf) {
          HCK(cudaMemcpyAsync(grown, logbuf, (size_t)sweeps * sweep_log * sizeof(double2),
                              cudaMemcpyDeviceToDevice, s.stream));
          HTRY(s.release(logbuf));
        }
        logbuf = grown;
        log_cap = cap;
      }
      HCK(cudaMemcpyAsync(logbuf + (size_t)sweeps * sweep_log, slots,
                          sweep_log * sizeof(double2), cudaMemcpyDeviceToDevice, s.stream));
    }
    HCK(cudaStreamSynchronize(s.stream));
    ++sweeps;
    done = true;
    for (int m = 0; m < n_mat; ++m) {
      const double off = s.host_norms[2 * m];
      if (!std::isfinite(off))
        return hfail(SWKB_ERR_INVALID_ARG, "matrix %d became non-finite", m);
      done = done && off <= kTol * kTol * fro[m];
    }
  }
  if (sweeps_out) *sweeps_out = sweeps;
  if (log) {
    log->d = logbuf;
    log->rounds = sweeps * (P - 1);
  }
  return SWKB_OK;
}

// v <- W^T v for vecs_per_mat vectors of P complex values per matrix
swkb_status replay_back(Scratch& s, const RotLog& log, int P, int n_mat, int vecs_per_mat,
                        double2* vecs) {
  const int npair = P / 2;
  const int threads = std::min(1024, std::max(32, (npair + 31) / 32 * 32));
  if ((npair + threads - 1) / threads > kReplayMaxPerThread)
    return hfail(SWKB_ERR_INVALID_ARG, "matrix too large for the rotation replay");
  const size_t smem = (size_t)P * sizeof(double2);
  if (smem > 48 * 1024)
    HCK(cudaFuncSetAttribute(k_replay, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_replay<<<n_mat * vecs_per_mat, threads, smem, s.stream>>>(log.d, log.rounds, P, n_mat,
                                                              vecs_per_mat, vecs);
  HCK(cudaGetLastError());
  return SWKB_OK;
}

swkb_status open_stream(Scratch& s, int on_device, void* user_stream) {
  // the caller's device work must be finished before the private stream reads it
  if (on_device) HCK(cudaStreamSynchronize((cudaStream_t)user_stream));
  HCK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
  return SWKB_OK;
}

swkb_status sym_eig(int batch, int n, const double* A_in, double* lam_out, double* vec_out,
                    int* sweeps_out, int on_device, void* user_stream) {
  if (!A_in || !lam_out) return hfail(SWKB_ERR_INVALID_ARG, "NULL matrix or eigenvalue array");
  if (batch < 1 || batch > 65535 || n < 1 || n > 8192)
    return hfail(SWKB_ERR_INVALID_ARG,
                 "batch %d, n %d: need 1 <= batch <= 65535 and 1 <= n <= 8192", batch, n);
  Scratch s;
  HTRY(open_stream(s, on_device, user_stream));
  const int P = n + (n & 1);
  const size_t nn = (size_t)n * n * batch, PP = (size_t)P * P * batch;
  double *A = nullptr, *W = nullptr, *src = nullptr, *lam = nullptr, *vec = nullptr;
  HTRY(s.alloc(&A, PP));
  if (vec_out) HTRY(s.alloc(&W, PP));   // eigenvectors accumulated only when wanted
  if (on_device) {
    src = (double*)A_in;
    lam = lam_out;
    vec = vec_out;
  } else {
    HTRY(s.alloc(&src, nn));
    HTRY(s.alloc(&lam, (size_t)n * batch));
    if (vec_out) HTRY(s.alloc(&vec, nn));
    HCK(cudaMemcpyAsync(src, A_in, nn * sizeof(double), cudaMemcpyHostToDevice, s.stream));
  }
  k_load_sym<<<grid_for((long long)PP), kThreads, 0, s.stream>>>(src, n, P, batch, A, W);
  HCK(cudaGetLastError());
  HTRY(jacobi(s, A, W, nullptr, P, batch, sweeps_out, nullptr));
  k_copy_leading<<<grid_for((long long)nn), kThreads, 0, s.stream>>>(A, W, n, P, batch, lam, vec);
  HCK(cudaGetLastError());
  if (!on_device) {
    HCK(cudaMemcpyAsync(lam_out, lam, (size_t)n * batch * sizeof(double),
                        cudaMemcpyDeviceToHost, s.stream));
    if (vec_out)
      HCK(cudaMemcpyAsync(vec_out, vec, nn * sizeof(double), cudaMemcpyDeviceToHost, s.stream));
  }
  HCK(cudaStreamSynchronize(s.stream));
  return SWKB_OK;
}

swkb_status hill_propagate(const swkb_hill_desc* d, int batch, const double* k,
                           const double* eps_in, const double* u0_in, int n_x, const double* x,
                           double* u_out, double* lam_out, int on_device, void* user_stream) {
  if (!d || !k || !eps_in || !u0_in || !x || !u_out)
    return hfail(SWKB_ERR_INVALID_ARG, "NULL argument");
  if (d->bc < SWKB_BC_PERIODIC || d->bc > SWKB_BC_DIRICHLET)
    return hfail(SWKB_ERR_INVALID_ARG, "unknown boundary condition %d", d->bc);
  if (batch < 1 || batch > 16384 || n_x < 1 || d->n_z < 2)
    return hfail(SWKB_ERR_INVALID_ARG, "need 1 <= batch <= 16384, n_x >= 1, n_z >= 2");
  if (!(d->z_b > d->z_a)) return hfail(SWKB_ERR_INVALID_ARG, "need z_b > z_a");
  FieldDims f;
  f.n_z = d->n_z;
  f.mirror = d->bc == SWKB_BC_NEUMANN ? 1 : (d->bc == SWKB_BC_DIRICHLET ? -1 : 0);
  f.N = f.mirror ? 2 * d->n_z : d->n_z;
  const double H = d->z_b - d->z_a;
  const double L = f.mirror ? 2.0 * H : H;
  const double dz = H / d->n_z;
  if (f.mirror) {
    f.m_c = d->n_z;
  } else {
    const double mc = (d->z_sym - d->z_a) / dz;
    f.m_c = (int)llround(mc);
    if (!(fabs(mc - f.m_c) <= 1e-9 * (1.0 + fabs(mc))) || f.m_c < 0 || f.m_c >= f.N)
      return hfail(SWKB_ERR_INVALID_ARG, "z_sym must be a field point inside [z_a, z_b)");
  }
  if (d->K < 1 || 2LL * d->K >= f.N)
    return hfail(SWKB_ERR_INVALID_ARG, "K = %d: need 1 <= K < N_period / 2 = %d", d->K, f.N / 2);
  if (d->n_q < 2 * d->K || d->n_q > (1 << 24))
    return hfail(SWKB_ERR_INVALID_ARG, "n_q = %d: need 2 K <= n_q <= 2^24", d->n_q);
  for (int b = 0; b < batch; ++b)
    if (!(k[b] > 0) || !std::isfinite(k[b]))
      return hfail(SWKB_ERR_INVALID_ARG, "k[%d] must be positive and finite", b);
  for (int r = 0; r < n_x; ++r)
    if (!(x[r] >= 0) || !std::isfinite(x[r]))
      return hfail(SWKB_ERR_INVALID_ARG, "x[%d] must be >= 0 and finite", r);
  HillDims hd;
  hd.K = d->K;
  hd.n_par = f.mirror ? 1 : 2;
  hd.par0 = f.mirror < 0 ? 1 : 0;
  hd.P = (d->K + 1) + ((d->K + 1) & 1);
  hd.kappa1 = 2.0 * M_PI / L;
  const int n_mat = batch * hd.n_par, P = hd.P, J = 2 * d->K + 1;
  const int n_eig = hd.n_par == 2 ? 2 * d->K + 1 : (hd.par0 ? d->K : d->K + 1);
  if (P > 8192 || (double)P * P * n_mat * sizeof(double) > 64e9)
    return hfail(SWKB_ERR_INVALID_ARG, "K or batch x K too large for one call");

  Scratch s;
  HTRY(open_stream(s, on_device, user_stream));
  const size_t n_eps = (size_t)batch * (d->n_q + 1), n_u = (size_t)batch * d->n_z;
  const size_t n_out = (size_t)batch * n_x * d->n_z;
  double *eps = nullptr, *kd = nullptr, *xd = nullptr, *tq = nullptr, *eh = nullptr;
  double *A = nullptr, *lam = nullptr;
  double2 *u0 = nullptr, *tab = nullptr, *uh = nullptr, *ph = nullptr, *out = nullptr;
  if (on_device) {
    eps = (double*)eps_in;
    u0 = (double2*)u0_in;
    out = (double2*)u_out;
    lam = lam_out;
  } else {
    HTRY(s.alloc(&eps, n_eps));
    HTRY(s.alloc(&u0, n_u));
    HTRY(s.alloc(&out, n_out));
    if (lam_out) HTRY(s.alloc(&lam, (size_t)batch * n_eig));
    HCK(cudaMemcpyAsync(eps, eps_in, n_eps * sizeof(double), cudaMemcpyHostToDevice, s.stream));
    HCK(cudaMemcpyAsync(u0, u0_in, n_u * sizeof(double2), cudaMemcpyHostToDevice, s.stream));
  }
  HTRY(s.alloc(&kd, batch));
  HTRY(s.alloc(&xd, n_x));
  HTRY(s.alloc(&tq, 2 * (size_t)d->n_q));
  HTRY(s.alloc(&tab, f.N));
  HTRY(s.alloc(&eh, (size_t)batch * J));
  HTRY(s.alloc(&A, (size_t)n_mat * P * P));
  HTRY(s.alloc(&uh, (size_t)n_mat * P));
  HTRY(s.alloc(&ph, (size_t)n_mat * n_x * P));
  HCK(cudaMemcpyAsync(kd, k, batch * sizeof(double), cudaMemcpyHostToDevice, s.stream));
  HCK(cudaMemcpyAsync(xd, x, n_x * sizeof(double), cudaMemcpyHostToDevice, s.stream));

  k_dct_table<<<grid_for(2LL * d->n_q), kThreads, 0, s.stream>>>(tq, d->n_q);
  k_period_table<<<grid_for(f.N), kThreads, 0, s.stream>>>(tab, f.N);
  k_eps_means<<<dim3(J, batch), kThreads, 0, s.stream>>>(eps, d->n_q, tq, J, eh);
  k_build<<<grid_for((long long)n_mat * P * P), kThreads, 0, s.stream>>>(hd, n_mat, kd, eh, A,
                                                                         nullptr);
  HCK(cudaGetLastError());
  // eigenvalues on the diagonal of A; the eigenvectors stay implicit, as the
  // logged rotations W = J_T^T ... J_1^T
  // the field's basis projections uh ride along the rotations: a = W uh
  k_project<<<dim3(P, n_mat), kThreads, 0, s.stream>>>(u0, f, hd, tab, uh);
  RotLog lg;
  HTRY(jacobi(s, A, nullptr, uh, P, n_mat, nullptr, &lg));
  k_advance_coefficients<<<grid_for((long long)n_mat * n_x * P), kThreads, 0, s.stream>>>(
      A, uh, hd, n_mat, xd, n_x, ph);                     // a_j exp(i alpha_j x)
  HTRY(replay_back(s, lg, P, n_mat, n_x, ph));           // g = W^T (a exp(i alpha x))
  k_synthesize<<<grid_for((long long)n_out), kThreads, 0, s.stream>>>(ph, f, hd, batch, n_x, tab,
                                                                       out);
  if (lam) k_eigenvalues<<<grid_for((long long)batch * n_eig), kThreads, 0, s.stream>>>(
      A, hd, batch, lam);
  HCK(cudaGetLastError());
  if (!on_device) {
    HCK(cudaMemcpyAsync(u_out, out, n_out * sizeof(double2), cudaMemcpyDeviceToHost, s.stream));
    if (lam_out)
      HCK(cudaMemcpyAsync(lam_out, lam, (size_t)batch * n_eig * sizeof(double),
                          cudaMemcpyDeviceToHost, s.stream));
  }
  HCK(cudaStreamSynchronize(s.stream));
  return SWKB_OK;
}

}  // namespace

extern "C" {

swkb_status swkb_sym_eig(int32_t batch, int32_t n, const double* A, double* lambda_out,
                         double* vectors_out, int32_t* sweeps_out, int32_t on_device,
                         void* cuda_stream) {
  try {
    int sw = 0;
    const swkb_status st =
        sym_eig(batch, n, A, lambda_out, vectors_out, &sw, on_device, cuda_stream);
    if (st == SWKB_OK && sweeps_out) *sweeps_out = sw;
    return st;
  } catch (...) {
    return hfail(SWKB_ERR_OOM, "host allocation failed");
  }
}

swkb_status swkb_hill_propagate(const swkb_hill_desc* desc, int32_t batch, const double* k,
                                const double* eps, const double* u0, int32_t n_x,
                                const double* x, double* u_out, double* lambda_out,
                                int32_t on_device, void* cuda_stream) {
  try {
    return hill_propagate(desc, batch, k, eps, u0, n_x, x, u_out, lambda_out, on_device,
                          cuda_stream);
  } catch (...) {
    return hfail(SWKB_ERR_OOM, "host allocation failed");
  }
}

}  // extern "C"
