// Persistent batch kernel of libswkb.so: many propagations of uneven size
// (frequency, N_z, range, medium) advanced screen by screen inside ONE
// cooperative launch that walks a device work queue.
//
// Work.  Every instance i runs the steps of Algorithm 1 on every screen s
// (s = 0 .. n_i - 1): the ray march (b), the two DFT passes (a), the landing
// brackets and the fused interpolation + modal sum (c, d); before the first
// screen its field is extended to the period, after the last one reduced
// (reflection, absorber) and written out.  Each step of each screen is a
// "job" of independent work items (groups of the standalone kernels' blocks);
// the queue lists the jobs of all instances interleaved step by step:
//
//   prologue   INIT(i), MARCH(i, 0)                             for every i
//   step s     OUTPUT(i finished at s - 1), FFT1(i, s),
//              MARCH(i, s + 1) for i = 0 mod 3, FFT2(i, s), BRACKET(i, s),
//              MARCH(i, s + 1) for i = 1 mod 3, RESUM(i, s),
//              MARCH(i, s + 1) for i = 2 mod 3, REDUCE(i finishing at s)
//   epilogue   OUTPUT(i finished last)
//
// so that every dependency of a job lies in an earlier job.  Rays depend on
// the medium only, so the march runs a screen ahead, into one of three
// ray-buffer sets (set s mod 3); MARCH(s + 1) waits for RESUM(s - 2), the
// set's last reader.  The other dependencies: FFT1(s) on RESUM(s - 1) (its
// partial sums are the field) or INIT; FFT2(s) on FFT1(s); BRACKET(s) on
// MARCH(s); RESUM(s) on FFT2(s) and BRACKET(s); REDUCE on the last RESUM;
// OUTPUT on REDUCE.  Monotonic counters per (instance, step kind, screen mod
// 3) count finished items; a job waits until its producers' counters reach
// their totals through that screen (screens sharing a counter are three
// apart, and the dependencies above order them).
//
// Execution.  A CTA claims the next item (an atomic per job; a shared job
// pointer advances past exhausted jobs), thread 0 waits for the item's
// dependencies (acquire loads of the counters, bounded: after the batch's
// wait limit the CTA raises the batch error and every CTA leaves), the CTA
// runs the item with the same device bodies as the standalone kernels, and
// thread 0 publishes it (fence, counter increment).  Items are claimed in
// queue order and all CTAs are co-resident (cooperative launch), so the
// oldest unfinished item always has its producers finished: the queue cannot
// deadlock, and no wait is unbounded.  Data produced inside the launch is
// read from L2 (ld.global.cg), never through the non-coherent path.
//
// Per instance the arithmetic, launch shapes and summation orders are those of
// its own plan, so every field equals the one the instance's plan computes
// alone, bit for bit.

#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "swkb.h"
#include "swkb_device.cuh"

namespace swkb {
namespace {

enum Phase {
  PH_INIT = 0, PH_MARCH, PH_FFT1, PH_FFT2, PH_BRACKET, PH_RESUM, PH_REDUCE, PH_OUTPUT, PH_COUNT
};
constexpr int kSets = 3;          // ray-buffer sets per instance
constexpr int kThreads = 256;
// standalone blocks per work item (small blocks are grouped so that an item
// is worth its claim)
constexpr int VB_INIT = 8, VB_MARCH = 2, VB_FFT1 = 4, VB_FFT2 = 8, VB_BRACKET = 64,
              VB_REDUCE = 8, VB_OUTPUT = 8;
// resummation blocks per item: one per 128-thread half of the CTA, or one in
// the lower half when two blocks' shared memory does not fit (Ctl.resum_per_item)

struct Job {
  int inst, phase, step, items;
  int dep_c[2];          // counter (inst * PH_COUNT + phase) * kSets + step mod kSets, or -1
  unsigned dep_need[2];  // finished items that counter must reach
};

template <typename T>
struct Inst {
  MarchArgs<T> march[kSets];       // stage row of screen 0 (patched per screen)
  BracketArgs<T> bracket[kSets];
  ResumArgs<T> resum[kSets];
  FftArgs<T> fft_fresh, fft_next;
  ReduceArgs<T> fin;
  const double* u0;                // n_z complex128 input
  double* out;                     // n_z complex128 output
  typename C2<T>::type* u;         // the plan's period field
  int n_z, N, mirror, q0, stage_rows, stage_stride, multi, cubic;
  int march_bx, march_blocks, bracket_bx, fft1_blocks, fft2_blocks, resum_blocks, resum_pw;
  int reduce_n, out_off;
};

struct Ctl {
  const Job* jobs;
  int n_jobs;
  unsigned* claimed;               // [n_jobs] items handed out
  unsigned* done;                  // [n_inst * PH_COUNT * kSets + 1] finished items (last: never)
  int* cur;                        // first job that may have unclaimed items
  unsigned* error;                 // 0, or 1: a wait gave up
  unsigned long long wait_ns;      // bound of every wait
  unsigned resum_slot;             // shared bytes of one resummation block
  int resum_per_item;              // 2, or 1 when two slots do not fit
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Thread 0: the next item (job index, item index in *item), or -1 when the
// queue is exhausted or the batch has failed.
__device__ int claim(const Ctl& c, int* item) {
  int j = *reinterpret_cast<volatile int*>(c.cur);
  while (j < c.n_jobs) {
    if (ld_volatile(c.error)) return -1;
    const unsigned b = atomicAdd(c.claimed + j, 1u);
    if (b < (unsigned)c.jobs[j].items) {
      *item = (int)b;
      return j;
    }
    atomicCAS(c.cur, j, j + 1);   // the job is exhausted: move the pointer on
    j = *reinterpret_cast<volatile int*>(c.cur);
  }
  return -1;
}

// Thread 0: wait until the job's producers have finished; false when the
// wait limit passed (the batch error is raised) or the batch failed.
__device__ bool wait_deps(const Ctl& c, const Job& jb) {
  const unsigned long long t0 = now_ns();
  for (int k = 0; k < 2; ++k) {
    if (jb.dep_c[k] < 0) continue;
    const unsigned* ctr = c.done + jb.dep_c[k];
    while (ld_acquire(ctr) < jb.dep_need[k]) {
      if (ld_volatile(c.error)) return false;
      if (now_ns() - t0 > c.wait_ns) {
        atomicCAS(c.error, 0u, 1u);
        return false;
      }
      __nanosleep(200);
    }
  }
  return true;
}

// Copy an argument block into shared memory (all threads; 8-byte words).
template <typename A>
__device__ __forceinline__ void stage_args(A* dst, const A* src, int tid) {
  static_assert(sizeof(A) % 8 == 0, "argument blocks are 8-byte multiples");
  for (int w = tid; w < (int)(sizeof(A) / 8); w += kThreads)
    reinterpret_cast<unsigned long long*>(dst)[w] =
        __ldg(reinterpret_cast<const unsigned long long*>(src) + w);
}

template <typename T>
__device__ __forceinline__ void march_item(const Inst<T>& I, int set, int step, int item,
                                           int tid) {
  MarchArgs<T> a = I.march[set];
  const int row = min(max(I.q0 + step, 0), I.stage_rows - 1);
  a.st.c += (long long)row * I.stage_stride;
  a.st.th += (long long)row * I.stage_stride;
  if constexpr (sizeof(T) == 4) {
    if (I.multi) {
      if (I.cubic) march_x2_body<true, false, true>(a, item, tid);
      else march_x2_body<true, false, false>(a, item, tid);
    } else {
      if (I.cubic) march_x2_body<false, false, true>(a, item, tid);
      else march_x2_body<false, false, false>(a, item, tid);
    }
  } else {
    const int bx = item % I.march_bx, by = item / I.march_bx;
    if (I.multi) march_body<T, true, false>(a, bx, by, tid & 31, tid >> 5);
    else march_body<T, false, false>(a, bx, by, tid & 31, tid >> 5);
  }
}

template <typename T>
__device__ __forceinline__ void resum_item(const ResumArgs<T>& r, int pw, int v, int tid,
                                           unsigned char* smem, int sub) {
  switch (pw) {
    case 2: resum_body<T, 2, LD_CG, 1>(r, v, tid, smem, sub); break;
    case 4: resum_body<T, 4, LD_CG, 1>(r, v, tid, smem, sub); break;
    case 8: resum_body<T, 8, LD_CG, 1>(r, v, tid, smem, sub); break;
    default: resum_body<T, 16, LD_CG, 1>(r, v, tid, smem, sub); break;
  }
}

union alignas(16) ArgSlot {
  BracketArgs<float> bf;
  BracketArgs<double> bd;
  ResumArgs<float> rf;
  ResumArgs<double> rd;
  FftArgs<float> ff;
  FftArgs<double> fd;
  ReduceArgs<float> gf;
  ReduceArgs<double> gd;
};

template <typename T> __device__ __forceinline__ BracketArgs<T>& slot_bracket(ArgSlot& s);
template <> __device__ __forceinline__ BracketArgs<float>& slot_bracket<float>(ArgSlot& s) { return s.bf; }
template <> __device__ __forceinline__ BracketArgs<double>& slot_bracket<double>(ArgSlot& s) { return s.bd; }
template <typename T> __device__ __forceinline__ ResumArgs<T>& slot_resum(ArgSlot& s);
template <> __device__ __forceinline__ ResumArgs<float>& slot_resum<float>(ArgSlot& s) { return s.rf; }
template <> __device__ __forceinline__ ResumArgs<double>& slot_resum<double>(ArgSlot& s) { return s.rd; }
template <typename T> __device__ __forceinline__ FftArgs<T>& slot_fft(ArgSlot& s);
template <> __device__ __forceinline__ FftArgs<float>& slot_fft<float>(ArgSlot& s) { return s.ff; }
template <> __device__ __forceinline__ FftArgs<double>& slot_fft<double>(ArgSlot& s) { return s.fd; }
template <typename T> __device__ __forceinline__ ReduceArgs<T>& slot_reduce(ArgSlot& s);
template <> __device__ __forceinline__ ReduceArgs<float>& slot_reduce<float>(ArgSlot& s) { return s.gf; }
template <> __device__ __forceinline__ ReduceArgs<double>& slot_reduce<double>(ArgSlot& s) { return s.gd; }

// FP32: 3 CTAs of 256 threads per SM (85 registers a thread); FP64: 1.
template <typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 3 : 1)
    k_batch(const Ctl c, const Inst<T>* __restrict__ insts) {
  using V = typename C2<T>::type;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_job, s_item;
  __shared__ ArgSlot s_args;
  __shared__ V s_wsum[2][FFT2_THREADS / 32];
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      int item = 0;
      int j = claim(c, &item);
      if (j >= 0 && !wait_deps(c, c.jobs[j])) j = -1;
      s_job = j;
      s_item = item;
    }
    __syncthreads();
    const int j = s_job;
    if (j < 0) break;
    const int item = s_item;
    const Job jb = c.jobs[j];
    const Inst<T>& I = insts[jb.inst];
    const int set = jb.step % kSets;
    switch (jb.phase) {
      case PH_INIT:
        for (int v = 0; v < VB_INIT; ++v)
          init_body<T>(I.u0, I.n_z, I.N, I.mirror, I.u, ((item * VB_INIT + v) << 8) + tid);
        break;
      case PH_MARCH:
        for (int v = item * VB_MARCH; v < min(item * VB_MARCH + VB_MARCH, I.march_blocks); ++v)
          march_item<T>(I, set, jb.step, v, tid);
        break;
      case PH_FFT1: {
        FftArgs<T>& f = slot_fft<T>(s_args);
        stage_args(&f, jb.step == 0 ? &I.fft_fresh : &I.fft_next, tid);
        __syncthreads();
        for (int v = item * VB_FFT1; v < min(item * VB_FFT1 + VB_FFT1, I.fft1_blocks); ++v) {
          fft1_body<T, LD_CG>(f, v, tid, smem);
          __syncthreads();   // the tile is reused by the next block
        }
        break;
      }
      case PH_FFT2: {
        FftArgs<T>& f = slot_fft<T>(s_args);
        stage_args(&f, jb.step == 0 ? &I.fft_fresh : &I.fft_next, tid);
        __syncthreads();
        const int sub = tid >> 7;
        for (int k = 0; k < VB_FFT2 / 2; ++k) {
          const int v = item * VB_FFT2 + 2 * k + sub;
          if (v < I.fft2_blocks) fft2_body<T, LD_CG, 1>(f, v, tid & 127, s_wsum[sub], sub);
          vb_sync<1>(sub);   // s_wsum is reused by the next mode
        }
        break;
      }
      case PH_BRACKET: {
        BracketArgs<T>& b = slot_bracket<T>(s_args);
        stage_args(&b, &I.bracket[set], tid);
        __syncthreads();
        const int nb = I.bracket_bx * (b.NRT - 1);
        for (int v = item * VB_BRACKET; v < min(item * VB_BRACKET + VB_BRACKET, nb); ++v)
          bracket_body<T, LD_CG>(b, v % I.bracket_bx, v / I.bracket_bx, tid);
        break;
      }
      case PH_RESUM: {
        ResumArgs<T>& r = slot_resum<T>(s_args);
        stage_args(&r, &I.resum[set], tid);
        __syncthreads();
        const int sub = tid >> 7;
        const int v = item * c.resum_per_item + sub;
        if (sub < c.resum_per_item && v < I.resum_blocks)
          resum_item<T>(r, I.resum_pw, v, tid & 127, smem + (size_t)sub * c.resum_slot, sub);
        break;
      }
      case PH_REDUCE: {
        ReduceArgs<T>& g = slot_reduce<T>(s_args);
        stage_args(&g, &I.fin, tid);
        __syncthreads();
        for (int v = 0; v < VB_REDUCE; ++v) {
          const int k = ((item * VB_REDUCE + v) << 8) + tid;
          if (k < I.reduce_n) reduce_body<T, LD_CG>(g, k);
        }
        break;
      }
      case PH_OUTPUT:
        for (int v = 0; v < VB_OUTPUT; ++v)
          output_body<T, LD_CG>(I.u, I.out_off, I.n_z, I.out, ((item * VB_OUTPUT + v) << 8) + tid);
        break;
      default:
        break;
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(c.done + (jb.inst * PH_COUNT + jb.phase) * kSets + jb.step % kSets, 1u);
    }
  }
}

int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace
}  // namespace swkb

using namespace swkb;

struct swkb_batch {
  int precision = SWKB_MIXED;
  int device = 0;
  int n = 0;
  std::vector<swkb_plan*> plans;
  std::vector<int> n_z, n_screens;
  std::vector<size_t> offset;          // complex values before instance i
  size_t total_nz = 0;
  std::vector<unsigned*> status;       // each plan's status word
  std::vector<void*> allocs;
  void* insts = nullptr;
  void* jobs = nullptr;
  unsigned* claimed = nullptr;
  unsigned* done = nullptr;
  int* cur = nullptr;
  unsigned* error = nullptr;
  double* in = nullptr;                // concatenated inputs (complex128)
  double* out = nullptr;               // concatenated outputs
  int n_jobs = 0, steps = 0;
  long long items = 0;
  int grid = 0, ctas_per_sm = 0;
  size_t smem = 0, resum_slot = 0, bytes = 0;
  int resum_per_item = 2;
  unsigned long long wait_ns = 2000000000ull;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph = nullptr;
  bool use_graph = true;
};

namespace {

swkb_status bfail(swkb_status s, const std::string& m) {
  swkb::set_last_error(m.c_str());
  return s;
}

#define BCK(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return bfail(SWKB_ERR_CUDA, std::string(#call " failed: ") + cudaGetErrorString(e_)); \
  } while (0)

#define TRY_B(x)                    \
  do {                              \
    swkb_status s_ = (x);           \
    if (s_ != SWKB_OK) return s_;   \
  } while (0)

swkb_status balloc(swkb_batch* b, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(SWKB_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  b->allocs.push_back(*p);
  b->bytes += bytes;
  return SWKB_OK;
}

void release(swkb_batch* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void* p : b->allocs) cudaFree(p);
  for (swkb_plan* p : b->plans) swkb_plan_destroy(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaSetDevice(cur);
  delete b;
}

template <typename T>
swkb_status build(swkb_batch* b, const swkb_request* reqs, const swkb_batch_options& opt) {
  using V = typename C2<T>::type;
  const int n = b->n;
  std::vector<Inst<T>> hi(n);
  std::vector<int> items((size_t)n * PH_COUNT);
  size_t resum_slot = 0, fft1_smem = 0;
  for (int i = 0; i < n; ++i) {
    PlanParts<T> pp;
    swkb_status st = plan_parts<T>(b->plans[i], &pp);
    if (st != SWKB_OK) return st;
    Inst<T>& I = hi[i];
    memset(&I, 0, sizeof(I));
    T* rd[kSets];
    T* rph[kSets];
    T* ra[kSets];
    int* jlo[kSets];
    int* jneg[kSets];
    for (int k = 0; k < kSets; ++k) {
      if (k < pp.sets) {
        rd[k] = pp.rd[k]; rph[k] = pp.rph[k]; ra[k] = pp.ra[k];
        jlo[k] = pp.jlo[k]; jneg[k] = pp.jneg[k];
        continue;
      }
      void* v;
      TRY_B(balloc(b, &v, pp.rays * sizeof(T))); rd[k] = (T*)v;
      TRY_B(balloc(b, &v, pp.rays * sizeof(T))); rph[k] = (T*)v;
      TRY_B(balloc(b, &v, pp.rays * sizeof(T))); ra[k] = (T*)v;
      TRY_B(balloc(b, &v, pp.jlo_n * sizeof(int))); jlo[k] = (int*)v;
      BCK(cudaMemsetAsync(jlo[k], 0, pp.jlo_n * sizeof(int), b->stream));
      jneg[k] = nullptr;
      if (pp.sym) {
        TRY_B(balloc(b, &v, pp.jlo_n * sizeof(int))); jneg[k] = (int*)v;
        BCK(cudaMemsetAsync(jneg[k], 0, pp.jlo_n * sizeof(int), b->stream));
      }
    }
    for (int k = 0; k < kSets; ++k) {
      I.march[k] = pp.march;
      I.march[k].out_d = rd[k]; I.march[k].out_ph = rph[k]; I.march[k].out_a = ra[k];
      I.bracket[k] = pp.bracket;
      I.bracket[k].d = rd[k]; I.bracket[k].jlo = jlo[k]; I.bracket[k].jlo_neg = jneg[k];
      I.resum[k] = pp.resum;
      I.resum[k].d = rd[k]; I.resum[k].ph = rph[k]; I.resum[k].a = ra[k];
      I.resum[k].jlo = jlo[k]; I.resum[k].jlo_neg = jneg[k];
    }
    I.fft_fresh = pp.fft_fresh;
    I.fft_next = pp.fft_next;
    I.fin = pp.fin;
    I.u0 = b->in + 2 * b->offset[i];
    I.out = b->out + 2 * b->offset[i];
    I.u = pp.u;
    I.n_z = pp.n_z; I.N = pp.N; I.mirror = pp.mirror; I.q0 = reqs[i].q0;
    I.stage_rows = pp.stage_rows; I.stage_stride = pp.stage_stride;
    I.multi = pp.n_cols > 1; I.cubic = pp.pieces > 0;
    I.march_bx = pp.march_bx; I.march_blocks = pp.march_blocks; I.bracket_bx = pp.bracket_bx;
    I.fft1_blocks = pp.fft1_blocks; I.fft2_blocks = pp.fft2_blocks;
    I.resum_blocks = pp.resum_blocks; I.resum_pw = pp.resum_pw;
    I.reduce_n = pp.reduce_n; I.out_off = pp.out_off;
    b->status[i] = pp.status;
    resum_slot = std::max(resum_slot, (pp.resum_smem + 15) & ~(size_t)15);
    fft1_smem = std::max(fft1_smem, pp.fft1_smem);
    int* it = &items[(size_t)i * PH_COUNT];
    it[PH_INIT] = cdiv(cdiv(pp.N, 256), VB_INIT);
    it[PH_MARCH] = cdiv(pp.march_blocks, VB_MARCH);
    it[PH_FFT1] = cdiv(pp.fft1_blocks, VB_FFT1);
    it[PH_FFT2] = cdiv(pp.fft2_blocks, VB_FFT2);
    it[PH_BRACKET] = cdiv((long long)pp.bracket_bx * (pp.NRT - 1), VB_BRACKET);
    it[PH_RESUM] = 0;   // set below, once the shared-memory budget is known
    it[PH_REDUCE] = cdiv(cdiv(pp.reduce_n, 256), VB_REDUCE);
    it[PH_OUTPUT] = cdiv(cdiv(pp.n_z, 256), VB_OUTPUT);
  }
  // resummation blocks per item (two in the CTA's halves when their shared
  // memory fits)
  {
    int optin = 0;
    BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    const size_t static_smem = sizeof(ArgSlot) + 1024;
    b->resum_per_item = 2 * resum_slot + static_smem <= (size_t)optin ? 2 : 1;
    for (int i = 0; i < n; ++i)
      items[(size_t)i * PH_COUNT + PH_RESUM] = cdiv(hi[i].resum_blocks, b->resum_per_item);
  }
  // the queue.  Finished items are counted per (instance, step kind, screen
  // mod 3): two screens of one kind that share a counter are three apart,
  // and the dependency chain keeps the later one from starting before the
  // earlier one has finished (MARCH(s + 3) waits for RESUM(s), which waits for
  // BRACKET(s) and FFT2(s), which wait for MARCH(s) and FFT1(s)), so a count
  // on a counter always counts whole screens in order.  (One counter per
  // kind would not: MARCH(s + 1) items may finish while MARCH(s) items run.)
  const int never = n * PH_COUNT * kSets;   // a counter nothing increments
  std::vector<Job> jobs;
  auto ctr = [](int i, int ph, int step) { return (i * PH_COUNT + ph) * kSets + step % kSets; };
  auto it = [&](int i, int ph) { return (long long)items[(size_t)i * PH_COUNT + ph]; };
  // items finished on the counter of screen s of kind ph once screen s is done
  auto upto = [&](int i, int ph, int s) { return (long long)(s / kSets + 1) * it(i, ph); };
  auto push = [&](int i, int ph, int step, int c0 = -1, long long n0 = 0, int c1 = -1,
                  long long n1 = 0) {
    Job j;
    j.inst = i; j.phase = ph; j.step = step; j.items = items[(size_t)i * PH_COUNT + ph];
    j.dep_c[0] = c0; j.dep_need[0] = (unsigned)n0;
    j.dep_c[1] = c1; j.dep_need[1] = (unsigned)n1;
    jobs.push_back(j);
  };
  int smax = 0;
  for (int i = 0; i < n; ++i) smax = std::max(smax, b->n_screens[i]);
  for (int i = 0; i < n; ++i) push(i, PH_INIT, 0);
  for (int i = 0; i < n; ++i) push(i, PH_MARCH, 0);
  // Each screen's chain FFT1 -> FFT2 -> RESUM -> next FFT1 is sequential per
  // instance, so independent work is placed between every producer and its
  // consumer: a third of the next screen's marches (by instance) after FFT1,
  // the brackets and another third after FFT2, the last third after RESUM
  // (the brackets of screen s then follow the marches of screen s by the
  // FFT1 and FFT2 segments).
  auto march_group = [&](int s, int g) {
    for (int i = g; i < n; i += 3) {
      const int m = s + 1;   // march a screen ahead into set m mod 3
      if (m < b->n_screens[i]) {
        if (m >= kSets)   // the set's last reader, RESUM(m - 3), is done
          push(i, PH_MARCH, m, ctr(i, PH_RESUM, m - kSets), upto(i, PH_RESUM, m - kSets));
        else
          push(i, PH_MARCH, m);
      }
    }
  };
  for (int s = 0; s <= smax; ++s) {
    for (int i = 0; i < n; ++i)   // reduced at the end of step s - 1
      if (s == b->n_screens[i])
        push(i, PH_OUTPUT, s, ctr(i, PH_REDUCE, s - 1), it(i, PH_REDUCE));
    if (s == smax) break;
    for (int i = 0; i < n; ++i)
      if (s < b->n_screens[i]) {
        if (s == 0) push(i, PH_FFT1, s, ctr(i, PH_INIT, 0), it(i, PH_INIT));
        else push(i, PH_FFT1, s, ctr(i, PH_RESUM, s - 1), upto(i, PH_RESUM, s - 1));
      }
    march_group(s, 0);
    for (int i = 0; i < n; ++i)
      if (s < b->n_screens[i]) push(i, PH_FFT2, s, ctr(i, PH_FFT1, s), upto(i, PH_FFT1, s));
    for (int i = 0; i < n; ++i)
      if (s < b->n_screens[i]) push(i, PH_BRACKET, s, ctr(i, PH_MARCH, s), upto(i, PH_MARCH, s));
    march_group(s, 1);
    for (int i = 0; i < n; ++i)
      if (s < b->n_screens[i])
        push(i, PH_RESUM, s, ctr(i, PH_FFT2, s), upto(i, PH_FFT2, s), ctr(i, PH_BRACKET, s),
             upto(i, PH_BRACKET, s));
    march_group(s, 2);
    for (int i = 0; i < n; ++i)
      if (s == b->n_screens[i] - 1)
        push(i, PH_REDUCE, s, ctr(i, PH_RESUM, s), upto(i, PH_RESUM, s));
  }
  // test hook: an item that waits on a counter nothing increments, so that
  // the bounded wait runs out (SWKB_BATCH_STALL=1)
  if (const char* e = getenv("SWKB_BATCH_STALL")) {
    if (e[0] == '1')
      for (Job& j : jobs)
        if (j.phase == PH_RESUM) {
          j.dep_c[1] = never;
          j.dep_need[1] = 1;
          break;
        }
  }
  b->steps = smax;
  b->n_jobs = (int)jobs.size();
  b->items = 0;
  for (const Job& j : jobs) b->items += j.items;
  BCK(cudaSetDevice(b->device));
  TRY_B(balloc(b, &b->insts, sizeof(Inst<T>) * n));
  BCK(cudaMemcpyAsync(b->insts, hi.data(), sizeof(Inst<T>) * n, cudaMemcpyHostToDevice, b->stream));
  TRY_B(balloc(b, &b->jobs, sizeof(Job) * jobs.size()));
  BCK(cudaMemcpyAsync(b->jobs, jobs.data(), sizeof(Job) * jobs.size(), cudaMemcpyHostToDevice,
                      b->stream));
  TRY_B(balloc(b, (void**)&b->claimed, sizeof(unsigned) * jobs.size()));
  TRY_B(balloc(b, (void**)&b->done, sizeof(unsigned) * (n * PH_COUNT * kSets + 1)));
  TRY_B(balloc(b, (void**)&b->cur, sizeof(int)));
  TRY_B(balloc(b, (void**)&b->error, sizeof(unsigned)));
  // launch shape: as many co-resident CTAs as fit (or as asked)
  b->resum_slot = resum_slot;
  int optin = 0, sms = 0, occ = 0;
  BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  const size_t static_smem = sizeof(ArgSlot) + 1024;
  b->smem = std::max((size_t)b->resum_per_item * resum_slot, fft1_smem);
  if (b->smem + static_smem > (size_t)optin)
    return bfail(SWKB_ERR_INVALID_ARG, "batch needs more shared memory per CTA than available");
  BCK(cudaFuncSetAttribute((const void*)k_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)b->smem));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch<T>, kThreads, b->smem));
  if (occ < 1) return bfail(SWKB_ERR_INVALID_ARG, "batch kernel does not fit on an SM");
  b->ctas_per_sm = opt.ctas_per_sm > 0 ? std::min(opt.ctas_per_sm, occ) : occ;
  b->grid = sms * b->ctas_per_sm;
  (void)sizeof(V);
  return SWKB_OK;
}

template <typename T>
swkb_status enqueue_run(swkb_batch* b) {
  Ctl c;
  c.jobs = (const Job*)b->jobs;
  c.n_jobs = b->n_jobs;
  c.claimed = b->claimed;
  c.done = b->done;
  c.cur = b->cur;
  c.error = b->error;
  c.wait_ns = b->wait_ns;
  c.resum_slot = (unsigned)b->resum_slot;
  c.resum_per_item = b->resum_per_item;
  BCK(cudaMemsetAsync(b->claimed, 0, sizeof(unsigned) * b->n_jobs, b->stream));
  BCK(cudaMemsetAsync(b->done, 0, sizeof(unsigned) * (b->n * PH_COUNT * kSets + 1), b->stream));
  BCK(cudaMemsetAsync(b->cur, 0, sizeof(int), b->stream));
  BCK(cudaMemsetAsync(b->error, 0, sizeof(unsigned), b->stream));
  const Inst<T>* insts = (const Inst<T>*)b->insts;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  BCK(cudaLaunchKernelEx(&cfg, k_batch<T>, c, insts));
  return SWKB_OK;
}

template <typename T>
swkb_status run_t(swkb_batch* b) {
  if (b->use_graph && !b->graph) {
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    swkb_status st = enqueue_run<T>(b);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->stream, &g);
    cudaGraphExec_t ex = nullptr;
    if (st == SWKB_OK && ec == cudaSuccess && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
      b->graph = ex;
    } else {
      // a capture the runtime refuses: launch directly from now on
      cudaGetLastError();
      b->use_graph = false;
    }
    if (g) cudaGraphDestroy(g);
  }
  if (b->graph) {
    BCK(cudaGraphLaunch(b->graph, b->stream));
    return SWKB_OK;
  }
  return enqueue_run<T>(b);
}

}  // namespace

extern "C" {

void swkb_batch_options_default(swkb_batch_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
}

swkb_status swkb_batch_create(int32_t n, const swkb_request* reqs,
                              const swkb_batch_options* opt_in, swkb_batch** out) {
  nvtxRangePushA("swkb_batch_create");
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  try {
    if (!out) return bfail(SWKB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || !reqs) return bfail(SWKB_ERR_INVALID_ARG, "need n >= 1 requests");
    swkb_batch_options opt;
    if (opt_in) opt = *opt_in; else swkb_batch_options_default(&opt);
    if (opt.ctas_per_sm < 0 || opt.wait_limit_ms < 0)
      return bfail(SWKB_ERR_INVALID_ARG, "ctas_per_sm and wait_limit_ms must be >= 0");
    swkb_batch* b = new swkb_batch();
    struct Guard { swkb_batch*& b; ~Guard() { if (b) release(b); } } guard{b};
    b->n = n;
    b->device = opt.device;
    if (opt.wait_limit_ms > 0) b->wait_ns = (unsigned long long)opt.wait_limit_ms * 1000000ull;
    const char* ge = getenv("SWKB_GRAPHS");
    b->use_graph = !(ge && ge[0] == '0');
    BCK(cudaSetDevice(b->device));
    if (opt.cuda_stream) {
      b->stream = (cudaStream_t)opt.cuda_stream;
    } else {
      BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
      b->own_stream = true;
    }
    for (int i = 0; i < n; ++i) {
      const swkb_request& r = reqs[i];
      if (!r.profile || !r.domain || !r.u0)
        return bfail(SWKB_ERR_INVALID_ARG, "request " + std::to_string(i) + ": NULL argument");
      if (r.n_screens < 1 || r.q0 < 0)
        return bfail(SWKB_ERR_INVALID_ARG,
                     "request " + std::to_string(i) + ": batched requests advance >= 1 screen");
      swkb_options o;
      if (r.options) o = *r.options; else swkb_options_default(&o);
      if (i == 0) b->precision = o.precision;
      if (o.precision != b->precision)
        return bfail(SWKB_ERR_INVALID_ARG, "all requests of a batch share one precision");
      o.cuda_stream = b->stream;
      o.device = b->device;
      o.reuse_rays = 0;
      o.planes = 0;
      swkb_plan* p = nullptr;
      swkb_status st = swkb_plan_create(r.profile, r.k, r.domain, r.n_z, r.screen_dx, &o, &p);
      if (st != SWKB_OK) {
        return bfail(st, "request " + std::to_string(i) + ": " + swkb_last_error());
      }
      b->plans.push_back(p);
      b->n_z.push_back(r.n_z);
      b->n_screens.push_back(r.n_screens);
      b->offset.push_back(b->total_nz);
      b->total_nz += (size_t)r.n_z;
    }
    b->status.assign(n, nullptr);
    TRY_B(balloc(b, (void**)&b->in, 2 * sizeof(double) * b->total_nz));
    TRY_B(balloc(b, (void**)&b->out, 2 * sizeof(double) * b->total_nz));
    for (int i = 0; i < n; ++i)
      BCK(cudaMemcpyAsync(b->in + 2 * b->offset[i], reqs[i].u0, 2 * sizeof(double) * b->n_z[i],
                          cudaMemcpyHostToDevice, b->stream));
    swkb_status st = b->precision == SWKB_FP64 ? build<double>(b, reqs, opt)
                                               : build<float>(b, reqs, opt);
    if (st != SWKB_OK) return st;
    BCK(cudaStreamSynchronize(b->stream));
    *out = b;
    b = nullptr;
    return SWKB_OK;
  } catch (const std::exception& e) {
    return bfail(SWKB_ERR_OOM, std::string("host allocation failed: ") + e.what());
  } catch (...) {
    return bfail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

swkb_status swkb_batch_run(swkb_batch* b, const double* u_in, double* u_out, int32_t on_device) {
  nvtxRangePushA("swkb_batch_run");
  struct Pop { ~Pop() { nvtxRangePop(); } } pop;
  try {
    if (!b) return bfail(SWKB_ERR_INVALID_ARG, "NULL batch");
    BCK(cudaSetDevice(b->device));
    const size_t nb = 2 * sizeof(double) * b->total_nz;
    if (u_in)
      BCK(cudaMemcpyAsync(b->in, u_in, nb,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          b->stream));
    TRY_B(b->precision == SWKB_FP64 ? run_t<double>(b) : run_t<float>(b));
    std::vector<unsigned> bits(b->n + 1, 0u);
    for (int i = 0; i < b->n; ++i)
      BCK(cudaMemcpyAsync(&bits[i], b->status[i], sizeof(unsigned), cudaMemcpyDeviceToHost,
                          b->stream));
    BCK(cudaMemcpyAsync(&bits[b->n], b->error, sizeof(unsigned), cudaMemcpyDeviceToHost,
                        b->stream));
    if (u_out)
      BCK(cudaMemcpyAsync(u_out, b->out, nb,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < b->n; ++i)
      if (bits[i]) BCK(cudaMemsetAsync(b->status[i], 0, sizeof(unsigned), b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (bits[b->n])
      return bfail(SWKB_ERR_TIMEOUT,
                   "a work item of the persistent batch kernel waited longer than the wait "
                   "limit for its producers; the launch was abandoned");
    for (int i = 0; i < b->n; ++i)
      if (bits[i]) {
        const swkb_status st = status_from_bits(bits[i]);
        return bfail(st, "request " + std::to_string(i) + ": " + swkb_last_error());
      }
    return SWKB_OK;
  } catch (...) {
    return bfail(SWKB_ERR_INVALID_ARG, "unexpected exception");
  }
}

swkb_status swkb_batch_get_info(const swkb_batch* b, swkb_batch_info* info) {
  if (!b || !info) return bfail(SWKB_ERR_INVALID_ARG, "NULL argument");
  memset(info, 0, sizeof(*info));
  info->instances = b->n;
  info->precision = b->precision;
  info->grid = b->grid;
  info->ctas_per_sm = b->ctas_per_sm;
  info->threads = kThreads;
  info->jobs = b->n_jobs;
  info->items = b->items;
  info->steps = b->steps;
  info->shared_bytes = b->smem;
  size_t bytes = b->bytes;
  for (swkb_plan* p : b->plans) bytes += plan_bytes(p);
  info->device_bytes = bytes;
  return SWKB_OK;
}

void swkb_batch_destroy(swkb_batch* b) { release(b); }

}  // extern "C"
