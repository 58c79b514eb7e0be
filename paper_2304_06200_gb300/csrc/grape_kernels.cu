// CUDA kernels (sm_103a) of the HG GRAPE evaluation.
//
// Work decomposition.  The n propagated columns (basis states psi_0^h) evolve
// independently (Sec. III.A: each column is its own forward-backward problem;
// only g = sum_h <phi_T^h|psi_N^h> and the gradient sum couple them).  Each
// column is owned by a "team" of CL CTAs (a thread-block cluster when CL > 1);
// the d rows are split into CL contiguous blocks of R rows, one per CTA, and one
// thread owns one row at a time.  Every Taylor term y = B x needs entries of x
// owned by other CTAs of the team: those are read from the owners' shared
// memory (distributed shared memory), and terms are separated by one team
// barrier (__syncthreads for CL = 1, barrier.cluster otherwise; with one row per
// thread its arrive and wait are split around the CTA-local entries).  Within a
// team nothing goes through global memory.  No kernel waits for another kernel or
// for a CTA outside its cluster: kernels are ordered by their streams and events.
//
// Row layout.  Each row of the union pattern holds its diagonal first (when every
// H_ii is real), then the entries whose B_ij is imaginary, then those whose B_ij
// is real, then the general ones; the one-row-per-thread loops apply the first
// three kinds with two multiplies instead of a complex multiply-add.
//
// Kernels
//   k_schedule        ||A_n||_1 = dt max_i sum_j |H_n,ij| and the (m_n, s_n) lookup (Sec. III.B, App. C)
//   k_forward         psi_n = (e^{B_n}_m)^s psi_{n-1}, C2 sum, C3 overlaps, checkpoints, psi_N, <phi_T|psi_N> partials
//   k_finalize        g, C1, C2, C3, C_amp, cost
//   k_costate         the costate chain alone, Horner vectors stored per block of steps (three-stage backward)
//   k_gradient        per-step gradient terms from the stored states and Horner vectors (three-stage backward)
//   k_backward        adjoint re-propagation of psi and the costate, gradient terms per step (one team per
//                     column; the fallback of the three-stage backward)
//   k_grad_reduce     sum of per-CTA gradient partials + amplitude-penalty gradient
//   k_sd_update       steepest-descent step u - (eta g) and the iterate's cost (Sec. II, Eq. (4))
//   k_check_finite    non-finite controls set the device error word
#include "grape_internal.h"

#include <algorithm>

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace grape {

// 1/q, 1/q! and (-1)^q / q! for q = 0..kMaxTaylor; 1/q as a pair of floats (hi, lo), hi + lo = 1/q to
// about 2^-48 (the compensated FP32 bulk)
__constant__ double c_inv_int[kMaxTaylor + 2];
__constant__ double c_inv_fact[kMaxTaylor + 2];
__constant__ double c_sgn_fact[kMaxTaylor + 2];
__constant__ float2 c_dw_inv[kMaxTaylor + 2];

static bool g_constants_ready[64] = {false};

static cudaError_t ensure_constants() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && g_constants_ready[dev]) return cudaSuccess;
  double inv_int[kMaxTaylor + 2], inv_fact[kMaxTaylor + 2], sgn_fact[kMaxTaylor + 2];
  inv_int[0] = 0.0;
  inv_fact[0] = 1.0;
  for (int q = 1; q < kMaxTaylor + 2; ++q) {
    inv_int[q] = 1.0 / q;
    inv_fact[q] = inv_fact[q - 1] / q;
  }
  for (int q = 0; q < kMaxTaylor + 2; ++q) sgn_fact[q] = (q & 1) ? -inv_fact[q] : inv_fact[q];
  float2 dw_inv[kMaxTaylor + 2];
  dw_inv[0] = make_float2(0.0f, 0.0f);
  for (int q = 1; q < kMaxTaylor + 2; ++q) {
    const float hi = (float)inv_int[q];
    dw_inv[q] = make_float2(hi, (float)(inv_int[q] - (double)hi));
  }
  e = cudaMemcpyToSymbol(c_dw_inv, dw_inv, sizeof(dw_inv));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_inv_int, inv_int, sizeof(inv_int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_inv_fact, inv_fact, sizeof(inv_fact));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sgn_fact, sgn_fact, sizeof(sgn_fact));
  if (e == cudaSuccess && dev >= 0 && dev < 64) g_constants_ready[dev] = true;
  return e;
}

// ------------------------------------------------------------------ complex helpers

__device__ __forceinline__ void cmac(double2& acc, const double2 a, const double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

__device__ __forceinline__ void cmac_conj(double2& acc, const double2 a, const double2 b) {  // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__device__ __forceinline__ double2 cmul(const double2 a, const double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cscale(const double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// ------------------------------------------------------------------ team barrier

template <bool CLUSTER>
__device__ __forceinline__ void team_sync() {
  if constexpr (CLUSTER) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
  } else {
    __syncthreads();
  }
}

// The two halves of the cluster barrier: work placed between them overlaps the barrier latency.
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Bulk asynchronous copy shared -> global of `bytes` (a multiple of 16, both addresses 16-byte
// aligned), issued by one thread.  Its writes go through the async proxy: a later release (e.g. the
// arrive of a cluster barrier) does not wait for them.  The source may be overwritten once
// bulk_wait_read has confirmed the copy read it.
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(ssrc));
  asm volatile("fence.proxy.async.shared::cta;\n\t"
               "cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n\t"
               "cp.async.bulk.commit_group;\n" ::"l"(gdst), "r"(s), "r"(bytes) : "memory");
}
// Each thread orders its own shared-memory writes before later async-proxy reads of them: every
// thread that wrote a bulk copy's source runs this before the barrier after which one thread
// issues the copy.
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// At most N of this thread's bulk copies may still be reading their sources.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;\n" ::"n"(N) : "memory");
}
// Every bulk copy of this thread has completed (its writes are performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// The split barrier of the one-row-per-thread term loops.  A team of one CTA needs neither half: the
// __syncthreads that ends every term already orders each buffer's writes before the next term's
// reads (and its reads before the writes two terms later).
template <bool CLUSTER>
__device__ __forceinline__ void split_arrive() {
  if constexpr (CLUSTER) cluster_arrive();
}
template <bool CLUSTER>
__device__ __forceinline__ void split_wait() {
  if constexpr (CLUSTER) cluster_wait();
}

// ------------------------------------------------------------------ block reductions (deterministic)

__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += red[w];
  __syncthreads();
  return t;  // valid in thread 0
}

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t = fmax(t, red[w]);
  __syncthreads();
  return t;
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// ------------------------------------------------------------------ schedule: norm and (m, s)

// ||A_n||_1 = dt * max_i sum_j |H_n,ij| on the union pattern (the 1-norm equals the infinity norm
// for Hermitian H, footnote to Eq. (norm inequality)).  rows_max: the largest row sum of H_n over
// rows [r0, r1) (valid in thread 0; +inf marks a non-finite sum), the controls of step n in s_u.
__device__ __forceinline__ double rows_max(const ScheduleParams& p, const double* s_u, int r0, int r1, double* red) {
  double rmax = 0.0;
  bool bad = false;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double rs = 0.0;
    for (int64_t e = p.rowptr[i]; e < p.rowptr[i + 1]; ++e) {
      double2 v = p.h0v[e];
      for (int c = p.ectr_ptr[e]; c < p.ectr_ptr[e + 1]; ++c) {
        const double uk = s_u[p.ectr_k[c]];
        const double2 hv = p.ectr_val[c];
        v.x = fma(uk, hv.x, v.x);
        v.y = fma(uk, hv.y, v.y);
      }
      rs += sqrt(v.x * v.x + v.y * v.y);
    }
    if (!(rs <= 1e300)) bad = true;   // NaN or inf
    rmax = fmax(rmax, rs);
  }
  if (bad) rmax = __longlong_as_double(0x7ff0000000000000LL);
  return block_max(rmax, red);
}

// The paper's rule for step n from its largest row sum mx: the smallest s, then the smallest m, with
// E_A(m, s) <= tau (the host's breakpoint table); stores (m, s) and ||A_n||_1.
__device__ __forceinline__ void pick_ms(const ScheduleParams& p, int n, double mx) {
  const double x = p.dt * mx;
  int m = 0, s = 0;
  if (!(x <= 1e300)) {
    set_error(p.err, kErrNonFinite);
  } else {
    int s0 = 1;
    if (p.b_cap > 0.0) s0 = min(max(1, (int)ceil(x / p.b_cap)), p.s_cap);
    for (int si = s0; si <= p.s_cap && s == 0; ++si) {
      if (p.table_smax[si - 1] >= x) {
        for (int mi = 1; mi <= p.m_cap; ++mi)
          if (p.table[(int64_t)(si - 1) * p.m_cap + (mi - 1)] >= x) { m = mi; s = si; break; }
      }
    }
    if (s == 0) set_error(p.err, kErrTol);
  }
  p.ms_m[n] = m;
  p.ms_s[n] = s;
  p.norm1[n] = x;
}

// The (m, s) of steps b, b + nb, b + 2 nb, ... of one problem, one block per step.
__device__ __forceinline__ void schedule_body(const ScheduleParams& p, const int b, const int nb) {
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  for (int n = b; n < p.N; n += nb) {
    __syncthreads();
    if (threadIdx.x < p.K) s_u[threadIdx.x] = p.u[(int64_t)threadIdx.x * p.N + n];
    __syncthreads();
    const double mx = rows_max(p, s_u, 0, p.dim, red);
    if (threadIdx.x == 0) pick_ms(p, n, mx);
  }
}

// Few steps with many entries each (a dense H): the rows of a step are split over blockIdx.y chunks;
// each block maxes its chunk's largest row sum into norm1[n] as FP64 bits (non-negative doubles order
// like their bit patterns; norm1 zeroed before), then k_schedule_pick applies the rule per step.
// The maximum does not depend on the order, so the schedule is the one-block-per-step kernel's.
__global__ void __launch_bounds__(256) k_schedule_rows(const __grid_constant__ ScheduleParams p, int rows_per) {
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  const int r0 = blockIdx.y * rows_per, r1 = min(p.dim, r0 + rows_per);
  for (int n = blockIdx.x; n < p.N; n += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < p.K) s_u[threadIdx.x] = p.u[(int64_t)threadIdx.x * p.N + n];
    __syncthreads();
    const double mx = rows_max(p, s_u, r0, r1, red);
    if (threadIdx.x == 0)
      atomicMax(reinterpret_cast<unsigned long long*>(p.norm1) + n, (unsigned long long)__double_as_longlong(mx));
  }
}

__global__ void k_schedule_pick(const __grid_constant__ ScheduleParams p) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += gridDim.x * blockDim.x)
    pick_ms(p, n, p.norm1[n]);
}

__global__ void __launch_bounds__(256) k_schedule(const __grid_constant__ ScheduleParams p) {
  schedule_body(p, blockIdx.x, gridDim.x);
}

// Schedules of many problems in one launch: problem blockIdx.y, its steps over blockIdx.x.
__global__ void __launch_bounds__(256) k_schedule_batch(const ScheduleParams* __restrict__ ps) {
  __shared__ ScheduleParams sp;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(ps + blockIdx.y);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
    for (int i = threadIdx.x; i < (int)(sizeof(ScheduleParams) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  schedule_body(sp, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ sweep helpers

// Bulk (Taylor-term) arithmetic type: double for the FP64 path, dw for the compensated FP32 bulk.
// States (psi, chi), the W accumulators and every reduction stay FP64.
struct dw {};   // tag: a real number as an unevaluated pair of floats hi + lo
template <typename T> struct CxT;
template <> struct CxT<double> { using t = double2; };
template <> struct CxT<dw> { using t = float4; };   // {hi.re, hi.im, lo.re, lo.im}
template <typename T> using cx = typename CxT<T>::t;
template <typename T> constexpr bool kF64 = sizeof(cx<T>) == 16 && !__is_same(T, dw);

__device__ __forceinline__ double fmaT(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ double2 to_d2(const double2 v) { return v; }
template <typename T> __device__ __forceinline__ cx<T> from_d2(const double2 v);
template <> __device__ __forceinline__ double2 from_d2<double>(const double2 v) { return v; }
template <typename C2> __device__ __forceinline__ C2 czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float4 czero<float4>() { return make_float4(0.0f, 0.0f, 0.0f, 0.0f); }

template <typename C2>
__device__ __forceinline__ void cmacT(C2& acc, const C2 a, const C2 b) {  // acc += a b
  acc.x = fmaT(a.x, b.x, acc.x);
  acc.x = fmaT(-a.y, b.y, acc.x);
  acc.y = fmaT(a.x, b.y, acc.y);
  acc.y = fmaT(a.y, b.x, acc.y);
}

template <typename C2>
__device__ __forceinline__ void cmac_conjT(C2& acc, const C2 a, const C2 b) {  // acc += conj(a) b
  acc.x = fmaT(a.x, b.x, acc.x);
  acc.x = fmaT(a.y, b.y, acc.x);
  acc.y = fmaT(a.x, b.y, acc.y);
  acc.y = fmaT(-a.y, b.x, acc.y);
}

// ------------------------------------------------------------------ compensated FP32 (double-word) arithmetic
//
// A real bulk number is an unevaluated pair of floats hi + lo (|lo| about 2^-24 |hi| at most once
// normalised), a complex one float4 {hi.re, hi.im, lo.re, lo.im}.  Row sums accumulate in a DwAcc:
// per component a running float sum s and a float compensation c, the compensated dot product of
// Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005): each
// product a b of pairs is the float product p = ah bh with its exact error fma(ah, bh, -p) plus the
// cross terms ah bl + al bh; p joins s by Knuth's TwoSum, whose exact addition error joins c with
// the product's error.  A sum is normalised once, by Dekker's Fast2Sum.  The float operations are
// the correctly rounded intrinsics, which the compiler does not contract into FMAs (TwoSum relies
// on each sum being rounded on its own).  The result carries about 2^-48 relative error per
// operation on the magnitudes involved, against 2^-53 for FP64, at FP32 instruction rates.
struct DwAcc {
  float sr, si, cr, ci;
};
__device__ __forceinline__ DwAcc acc_zero() { return DwAcc{0.0f, 0.0f, 0.0f, 0.0f}; }

// (s, c) += p + e, p a float, e its small companion
__device__ __forceinline__ void acc_add(float& s, float& c, float p, float e) {
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  c = __fadd_rn(c, __fadd_rn(err, e));
  s = t;
}
// (s, c) += (ah + al)(bh + bl)
__device__ __forceinline__ void acc_mul(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  acc_add(s, c, p, e);
}
__device__ __forceinline__ void cmacT(DwAcc& a, const float4 v, const float4 x) {   // a += v x
  acc_mul(a.sr, a.cr, v.x, v.z, x.x, x.z);
  acc_mul(a.sr, a.cr, -v.y, -v.w, x.y, x.w);
  acc_mul(a.si, a.ci, v.x, v.z, x.y, x.w);
  acc_mul(a.si, a.ci, v.y, v.w, x.x, x.z);
}
__device__ __forceinline__ void cmac_conjT(DwAcc& a, const float4 v, const float4 x) {   // a += conj(v) x
  acc_mul(a.sr, a.cr, v.x, v.z, x.x, x.z);
  acc_mul(a.sr, a.cr, v.y, v.w, x.y, x.w);
  acc_mul(a.si, a.ci, v.x, v.z, x.y, x.w);
  acc_mul(a.si, a.ci, -v.y, -v.w, x.x, x.z);
}
// the normalised pair of each component (Fast2Sum)
__device__ __forceinline__ float4 dw_norm(const DwAcc& a) {
  const float hr = __fadd_rn(a.sr, a.cr), hi = __fadd_rn(a.si, a.ci);
  return make_float4(hr, hi, __fsub_rn(a.cr, __fsub_rn(hr, a.sr)), __fsub_rn(a.ci, __fsub_rn(hi, a.si)));
}
// x f for a complex pair x and a real pair f
__device__ __forceinline__ float4 dw_scale(const float4 x, const float2 f) {
  DwAcc a = acc_zero();
  acc_mul(a.sr, a.cr, x.x, x.z, f.x, f.y);
  acc_mul(a.si, a.ci, x.y, x.w, f.x, f.y);
  return dw_norm(a);
}
// a - b for complex pairs
__device__ __forceinline__ float4 dw_sub(const float4 a, const float4 b) {
  DwAcc r{a.x, a.y, a.z, a.w};
  acc_add(r.sr, r.cr, -b.x, -b.z);
  acc_add(r.si, r.ci, -b.y, -b.w);
  return dw_norm(r);
}
// a += (0, b) x: B_ij imaginary (H_ij real), b = the imaginary pair (v.y, v.w) of the stored value
__device__ __forceinline__ void dw_mac_imag(DwAcc& a, const float4 v, const float4 x) {
  acc_mul(a.sr, a.cr, -v.y, -v.w, x.y, x.w);
  acc_mul(a.si, a.ci, v.y, v.w, x.x, x.z);
}
// a += (b, 0) x: B_ij real (H_ij imaginary), b = the real pair (v.x, v.z)
__device__ __forceinline__ void dw_mac_real(DwAcc& a, const float4 v, const float4 x) {
  acc_mul(a.sr, a.cr, v.x, v.z, x.x, x.z);
  acc_mul(a.si, a.ci, v.x, v.z, x.y, x.w);
}
// acc += x for a complex pair x
__device__ __forceinline__ void acc_add4(DwAcc& a, const float4 x) {
  acc_add(a.sr, a.cr, x.x, x.z);
  acc_add(a.si, a.ci, x.y, x.w);
}
template <> __device__ __forceinline__ float4 from_d2<dw>(const double2 v) {
  const float hr = __double2float_rn(v.x), hi = __double2float_rn(v.y);
  return make_float4(hr, hi, __double2float_rn(v.x - (double)hr), __double2float_rn(v.y - (double)hi));
}
__device__ __forceinline__ double2 to_d2(const float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
__device__ __forceinline__ double2 to_d2(const DwAcc& a) {
  return make_double2((double)a.sr + (double)a.cr, (double)a.si + (double)a.ci);
}
// accumulator type of a bulk row sum
template <typename T> struct AccT { using t = cx<T>; };
template <> struct AccT<dw> { using t = DwAcc; };
template <typename T> using acc_t = typename AccT<T>::t;
template <typename T> __device__ __forceinline__ acc_t<T> acc0();
template <> __device__ __forceinline__ double2 acc0<double>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ DwAcc acc0<dw>() { return acc_zero(); }
// the bulk value of a row sum
__device__ __forceinline__ double2 finish(const double2 a) { return a; }
__device__ __forceinline__ float4 finish(const DwAcc& a) { return dw_norm(a); }

// One Horner step in bulk precision: chi/(p+1)! - yw (for FP64 in one fused rounding).
__device__ __forceinline__ double2 horner(const double2 ch, double f, const double2 yw) {
  return make_double2(fma(ch.x, f, -yw.x), fma(ch.y, f, -yw.y));
}

// B_ii x with B_ii = (0, b) imaginary (H_ii real): two multiplies.  As the first term of a row sum it
// equals the complex multiply-add on a zero accumulator.
__device__ __forceinline__ double2 diag_mul(double b, const double2 x) { return make_double2(-b * x.y, b * x.x); }
// y += (0, b) x and y += (b, 0) x: an imaginary or a real B_ij in two fused multiply-adds
__device__ __forceinline__ void mac_imag(double2& y, double b, const double2 x) {
  y.x = fma(-b, x.y, y.x);
  y.y = fma(b, x.x, y.y);
}
__device__ __forceinline__ void mac_real(double2& y, double b, const double2 x) {
  y.x = fma(b, x.x, y.x);
  y.y = fma(b, x.y, y.y);
}

template <typename T>
struct Carve {
  cx<T>* xb;          // exchange buffers (local)
  double2* psi;
  double2* chi;
  double2* inc;
  cx<T>* vals;
  double2* W;         // FP64 accumulators of conj(w_p) x_p per local entry
  DwAcc* Wb;          // compensated FP32 bulk: per-substep compensated staging of W
  cx<T>* wsm;         // Horner slots in shared memory (first m_smem)
  cx<T>* wgl;         // Horner slots in global scratch (slots >= m_smem)
  int* lrow;
  uint32_t* lcol;
};

template <typename T>
__device__ __forceinline__ Carve<T> carve(unsigned char* smem, const SweepParams& p, bool backward, int part) {
  const SmemLayout L = make_layout(backward, p.R, p.max_nnz_loc, p.in_smem, p.m_smem, (int)sizeof(cx<T>), !kF64<T>);
  double2* scr = p.scratch + (int64_t)part * p.scratch_stride;
  Carve<T> c;
  c.xb = reinterpret_cast<cx<T>*>(smem + L.xbuf);
  c.psi = reinterpret_cast<double2*>(smem + L.psi);
  c.chi = backward ? reinterpret_cast<double2*>(smem + L.chi) : nullptr;
  c.inc = reinterpret_cast<double2*>(smem + L.inc);
  c.vals = L.vals >= 0 ? reinterpret_cast<cx<T>*>(smem + L.vals) : reinterpret_cast<cx<T>*>(scr + p.scr_vals);
  c.W = L.W >= 0 ? reinterpret_cast<double2*>(smem + L.W) : scr + p.scr_W;
  c.Wb = L.Wb >= 0 ? reinterpret_cast<DwAcc*>(smem + L.Wb) : reinterpret_cast<DwAcc*>(scr + p.scr_Wb);
  c.wsm = L.wslot >= 0 ? reinterpret_cast<cx<T>*>(smem + L.wslot) : nullptr;
  c.wgl = reinterpret_cast<cx<T>*>(scr + p.scr_wslot);
  c.lrow = reinterpret_cast<int*>(smem + L.lrow);
  c.lcol = reinterpret_cast<uint32_t*>(smem + L.lcol);
  return c;
}

// Table of generic pointers to one exchange buffer of every CTA of the team.
template <typename T>
struct XTab {
  cx<T>* ptr[kMaxCluster];
};

// Assemble B_n = -i dt H_n / s on the CTA's local entries: vals[e] = (dt/s) * (-i) * (h0 + sum_k u_kn h_k),
// evaluated in FP64 and stored in the bulk precision.
template <typename T>
__device__ __forceinline__ void assemble(const SweepParams& p, cx<T>* vals, int64_t e0, int nnz_loc, double scale,
                                         const double* s_u) {
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) {
    const int64_t ge = e0 + e;
    double2 v = p.h0v[ge];
    for (int k = p.ectr_ptr[ge]; k < p.ectr_ptr[ge + 1]; ++k) {
      const double uk = s_u[p.ectr_k[k]];
      const double2 hv = p.ectr_val[k];
      v.x = fma(uk, hv.x, v.x);
      v.y = fma(uk, hv.y, v.y);
    }
    vals[e] = from_d2<T>(make_double2(scale * v.y, -scale * v.x));   // -i v
  }
}

// Entry ea of local row i is the row's diagonal (stored first when every H_ii is real).
__device__ __forceinline__ bool diag_at(const SweepParams& p, const uint32_t* lcol, int ea, int eb, int rank, int i) {
  return p.diag_first && ea < eb && (lcol[ea] & ~kCtrlBit) == (((uint32_t)rank << kOwnerShift) | (uint32_t)i);
}

// Segments of a row after its diagonal: [ea, *ci) imaginary B_ij, [*ci, *cr) real B_ij, the rest general.
__device__ __forceinline__ void row_segments(const uint32_t* lcol, int ea, int eb, int* ci, int* cr) {
  int e = ea;
  while (e < eb && (lcol[e] & kImagBBit)) ++e;
  *ci = e;
  while (e < eb && (lcol[e] & kRealBBit)) ++e;
  *cr = e;
}

// psi_n of column col in the segment buffer (slot (n / seg_M) % 2, position n % seg_M).
__device__ __forceinline__ double2* seg_state(const SweepParams& p, int n, int col) {
  const int pos = ((n / p.seg_M) & 1) * p.seg_M + n % p.seg_M;
  return p.seg + ((int64_t)pos * p.n_states + col) * p.dim;
}

__device__ __forceinline__ void load_controls(const SweepParams& p, int n, double* s_u) {
  if (threadIdx.x < p.K) s_u[threadIdx.x] = p.u[(int64_t)threadIdx.x * p.N + n];
}

template <typename T, bool CLUSTER>
__device__ __forceinline__ cx<T> xload(const cx<T>* local, const XTab<T>& tab, uint32_t enc) {
  if constexpr (CLUSTER) {
    return tab.ptr[(enc >> kOwnerShift) & 0xFFu][enc & kLocalMask];
  } else {
    return local[enc & kLocalMask];
  }
}


// Row products on the local pattern, returned as the row sum's bulk value.  FP64: one accumulator per
// chain (the FP64 pipe is the bound, so no extra instructions).  Compensated FP32 (latency bound):
// entries two at a time, both loads (a remote row costs a distributed-shared-memory round trip)
// issued before the two multiply-adds, which go to two accumulators.  The trip count is exact
// either way: no padded multiply-adds.
template <typename T, bool CLUSTER>
__device__ __forceinline__ cx<T> row_mv(const cx<T>* __restrict__ vals, const uint32_t* __restrict__ lcol, int ea,
                                        int eb, const cx<T>* xs, const XTab<T>& tab) {
  using C2 = cx<T>;
  if constexpr (kF64<T>) {
    C2 y = czero<C2>();
    for (int e = ea; e < eb; ++e) cmacT(y, vals[e], xload<T, CLUSTER>(xs, tab, lcol[e]));
    return y;
  } else {
    DwAcc y0 = acc_zero(), y1 = acc_zero();
    int e = ea;
    for (; e + 2 <= eb; e += 2) {
      const C2 v0 = vals[e], v1 = vals[e + 1];
      const C2 x0 = xload<T, CLUSTER>(xs, tab, lcol[e]);
      const C2 x1 = xload<T, CLUSTER>(xs, tab, lcol[e + 1]);
      cmacT(y0, v0, x0);
      cmacT(y1, v1, x1);
    }
    if (e < eb) cmacT(y0, vals[e], xload<T, CLUSTER>(xs, tab, lcol[e]));
    acc_add(y0.sr, y0.cr, y1.sr, y1.cr);
    acc_add(y0.si, y0.ci, y1.si, y1.ci);
    return dw_norm(y0);
  }
}

// Two chains through the same matrix row: ya = row . xa, yw = row . xw.
template <typename T, bool CLUSTER>
__device__ __forceinline__ void row_mv2(const cx<T>* __restrict__ vals, const uint32_t* __restrict__ lcol, int ea, int eb,
                                        const cx<T>* xa, const XTab<T>& ta, const cx<T>* xw, const XTab<T>& tw,
                                        cx<T>& ya, cx<T>& yw) {
  using C2 = cx<T>;
  if constexpr (kF64<T>) {
    C2 a = czero<C2>(), w = czero<C2>();
    for (int e = ea; e < eb; ++e) {
      const uint32_t enc = lcol[e];
      const C2 v = vals[e];
      cmacT(a, v, xload<T, CLUSTER>(xa, ta, enc));
      cmacT(w, v, xload<T, CLUSTER>(xw, tw, enc));
    }
    ya = a;
    yw = w;
  } else {
    DwAcc a = acc_zero(), w = acc_zero();
    for (int e = ea; e < eb; ++e) {
      const uint32_t enc = lcol[e];
      const C2 v = vals[e];
      const C2 x0 = xload<T, CLUSTER>(xa, ta, enc);
      const C2 x1 = xload<T, CLUSTER>(xw, tw, enc);
      cmacT(a, v, x0);
      cmacT(w, v, x1);
    }
    ya = dw_norm(a);
    yw = dw_norm(w);
  }
}

__device__ __forceinline__ void sweep_setup(const SweepParams& p, int* lrow, uint32_t* lcol, int r0, int nrows,
                                            int64_t e0, int nnz_loc) {
  for (int i = threadIdx.x; i <= nrows; i += blockDim.x) lrow[i] = (int)(p.rowptr[r0 + i] - e0);
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) lcol[e] = p.colenc[e0 + e];
}

// Everything one CTA of a team needs inside the sweeps.
template <typename T, bool CLUSTER>
struct Team {
  Carve<T> c;
  XTab<T>* tab;         // shared-memory table per exchange buffer
  // exchange buffer b (A chain 0,1; Horner chain 2,3; x chain 4,5), contiguous in shared memory
  __device__ __forceinline__ cx<T>* X(int b) const { return c.xb + b * R; }
  int r0, nrows, R, rank, CL;
  int64_t e0;
  int nnz_loc;
  // One row per thread (FP64 cluster teams): the thread's general entries are [ea, eb), those with a
  // column in this CTA's rows are the run [la, la + nloc) (their columns ascend, so do their owners),
  // and l1 = the smallest nloc of the warp's rows: the first l1 of the run are summed before the wait
  // of the cluster barrier, the other entries in one loop after it.
  // A diagonal stored first (entry ed, else -1) and the single-phase entries [c0, ci) (imaginary
  // B_ij) and [ci, ea) (real B_ij) precede [ea, eb): they are applied with two multiplies.
  bool one_row;
  int ea, eb, la, l1, ed, c0, ci;
};

// ------------------------------------------------------------------ forward sweep

// psi_n = (e^{B}_m)^s psi_{n-1} by the recursions b_j = (B/j) b_{j-1} (App. C Eq. (recursive relation 1))
// and c_l = e^B_m c_{l-1} (Eq. (recursive relation2)); C2 accumulates <psi_n|Omega|psi_n> (App. A).
// The state psi and the per-substep sum of the terms are FP64; the terms themselves use the bulk type.
// FP64 terms are kept unscaled, x_j = B^j c_{l-1} = j! b_j, and the sum takes x_j / j! in one fused
// multiply-add (one FP64 operation per component fewer than scaling every term by 1/j); FP32 terms
// keep the 1/j scaling, which bounds their range.
// The sweep of CTA `part` (team part / CL, rank part % CL); k_forward runs it for blockIdx.x, the
// batch work queue (k_queue) for one (problem, column) item at a time.
template <typename T, bool CLUSTER>
__device__ __forceinline__ void forward_body(const SweepParams& p, const int part) {
  using C2 = cx<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<T> tab[2];
  const int team = part / p.CL, rank = part % p.CL;
  const int r0 = min(rank * p.R, p.dim), r1 = min(r0 + p.R, p.dim), nrows = r1 - r0;
  const int64_t e0 = p.rowptr[r0];
  const int nnz_loc = (int)(p.rowptr[r1] - e0);
  const Carve<T> c = carve<T>(smem, p, false, part);
  C2* const X0 = c.xb;
  const int R = p.R;
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL) {
      tab[0].ptr[threadIdx.x] = cl.map_shared_rank(X0, threadIdx.x);
      tab[1].ptr[threadIdx.x] = cl.map_shared_rank(X0 + R, threadIdx.x);
    }
  }
  sweep_setup(p, c.lrow, c.lcol, r0, nrows, e0, nnz_loc);
  const int64_t col0 = (int64_t)team * p.dim + r0;
  // Segment recompute: steps [n_begin, n_end) from the segment's first state rec_src, every state of
  // the segment written to its slot of the segment buffer; no cost partials, checkpoints or psi_N.
  const bool rec = p.recompute != 0;
  const double2* const src0 = rec ? p.rec_src : p.psi0;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) c.psi[i] = src0[col0 + i];
  if (rec) {
    double2* const sg = seg_state(p, p.n_begin, team) + r0;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) sg[i] = c.psi[i];
  }
  double c2acc = 0.0;
  const bool split_rows = nrows <= (int)blockDim.x;   // one row per thread: split-barrier term loop
  // The thread's row: a diagonal stored first (ed), the single-phase entries [c0, ci) (imaginary B_ij)
  // and [ci, ea) (real B_ij), applied with two multiplies each, then the general entries [ea, eb), of
  // which [la, lb) have their column in this CTA's rows (the general entries' columns ascend, and so
  // do their owners, so these are contiguous).
  int ea = 0, eb = 0, la = 0, lb = 0, ed = -1, c0 = 0, ci = 0;
  __syncthreads();   // the local pattern written by sweep_setup
  if (split_rows && (int)threadIdx.x < nrows) {
    ea = c.lrow[threadIdx.x];
    eb = c.lrow[threadIdx.x + 1];
    if (diag_at(p, c.lcol, ea, eb, rank, threadIdx.x)) ed = ea++;
    c0 = ea;
    row_segments(c.lcol, c0, eb, &ci, &ea);
    la = ea;
    while (la < eb && ((c.lcol[la] >> kOwnerShift) & 0xFFu) < (uint32_t)rank) ++la;
    lb = la;
    while (lb < eb && ((c.lcol[lb] >> kOwnerShift) & 0xFFu) == (uint32_t)rank) ++lb;
  }
  team_sync<CLUSTER>();
  for (int n = rec ? p.n_begin : 0; n < (rec ? p.n_end : p.N); ++n) {
    const int m = p.ms_m[n], s = p.ms_s[n];
    if (s <= 0 || m <= 0) continue;   // flagged by k_schedule; uniform over the team
    load_controls(p, n, s_u);
    __syncthreads();
    assemble<T>(p, c.vals, e0, nnz_loc, p.dt / s, s_u);
    __syncthreads();
    for (int l = 0; l < s; ++l) {
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        X0[i] = from_d2<T>(c.psi[i]);
        c.inc[i] = make_double2(0.0, 0.0);   // the compensated bulk keeps a DwAcc in the same 16 bytes
      }
      if constexpr (kF64<T>) {
        if (split_rows) {
          // Each term: the entries whose column lies in this CTA's rows are summed between the
          // arrive and the wait of the previous term's cluster barrier; the remote ones after it.
          // X_q goes to buffer q & 1, which the other CTAs last read (as X_{q-2}) before they
          // arrived at barrier q-1, so writing it after wait(q-1) is safe; the last term of the
          // substep closes with a full barrier before X_0 of the next substep is written.
          __syncthreads();
          split_arrive<CLUSTER>();
          const int i = threadIdx.x;
          for (int q = 1; q <= m; ++q) {
            const int src = (q - 1) & 1, dst = q & 1;
            const C2* xs = X0 + src * R;
            C2 y = czero<C2>();
            if (i < nrows) {
              if (ed >= 0) y = diag_mul(c.vals[ed].y, xs[i]);
              for (int e = la; e < lb; ++e) cmacT(y, c.vals[e], xs[c.lcol[e] & kLocalMask]);
            }
            split_wait<CLUSTER>();
            if (i < nrows) {
              for (int e = c0; e < ci; ++e) {
                const uint32_t enc = c.lcol[e];
                mac_imag(y, c.vals[e].y, xload<T, CLUSTER>(xs, tab[src], enc));
              }
              for (int e = ci; e < ea; ++e) {
                const uint32_t enc = c.lcol[e];
                mac_real(y, c.vals[e].x, xload<T, CLUSTER>(xs, tab[src], enc));
              }
              // one loop over the remote entries on both sides of the local run, so that a warp
              // pays for its longest remote list once
              const int nl = la - ea, nr = nl + (eb - lb);
              for (int k = 0; k < nr; ++k) {
                const int e = k < nl ? ea + k : lb + (k - nl);
                const uint32_t enc = c.lcol[e];
                cmacT(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], enc));
              }
              X0[dst * R + i] = y;   // B^q c (unscaled)
              double2 a = c.inc[i];
              const double fq = c_inv_fact[q];
              a.x = fma(y.x, fq, a.x);
              a.y = fma(y.y, fq, a.y);
              c.inc[i] = a;
            }
            if (q < m) {
              __syncthreads();
              split_arrive<CLUSTER>();
            } else {
              team_sync<CLUSTER>();
            }
          }
          for (int j = threadIdx.x; j < nrows; j += blockDim.x) {
            double2 v = c.psi[j];
            const double2 a = c.inc[j];
            v.x += a.x;
            v.y += a.y;
            c.psi[j] = v;
          }
          continue;
        }
      } else {
        if (split_rows) {
          // The compensated bulk's term loop with the same split cluster barrier: scaled terms
          // b_q = (B b_{q-1}) / q, their sum kept in a register accumulator of the thread's row.
          __syncthreads();
          split_arrive<CLUSTER>();
          const int i = threadIdx.x;
          DwAcc incr = acc_zero();
          for (int q = 1; q <= m; ++q) {
            const int src = (q - 1) & 1, dst = q & 1;
            const C2* xs = X0 + src * R;
            DwAcc y = acc_zero();
            if (i < nrows) {
              if (ed >= 0) dw_mac_imag(y, c.vals[ed], xs[i]);
              for (int e = la; e < lb; ++e) cmacT(y, c.vals[e], xs[c.lcol[e] & kLocalMask]);
            }
            split_wait<CLUSTER>();
            if (i < nrows) {
              for (int e = c0; e < ci; ++e) dw_mac_imag(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              for (int e = ci; e < ea; ++e) dw_mac_real(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              const int nl = la - ea, nr = nl + (eb - lb);
              for (int k = 0; k < nr; ++k) {
                const int e = k < nl ? ea + k : lb + (k - nl);
                cmacT(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              }
              const C2 b = dw_scale(dw_norm(y), c_dw_inv[q]);
              X0[dst * R + i] = b;
              acc_add4(incr, b);
            }
            if (q < m) {
              __syncthreads();
              split_arrive<CLUSTER>();
            } else {
              team_sync<CLUSTER>();
            }
          }
          if (i < nrows) {
            const double2 a = to_d2(incr);
            double2 v = c.psi[i];
            v.x += a.x;
            v.y += a.y;
            c.psi[i] = v;
          }
          continue;
        }
      }
      team_sync<CLUSTER>();
      for (int q = 1; q <= m; ++q) {
        const int src = (q - 1) & 1, dst = q & 1;
        const double fq = c_inv_fact[q];
        const C2* xs = X0 + src * R;
        C2* xd = X0 + dst * R;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          C2 y = row_mv<T, CLUSTER>(c.vals, c.lcol, c.lrow[i], c.lrow[i + 1], xs, tab[src]);
          if constexpr (kF64<T>) {   // B^q c unscaled; the sum takes 1/q!
            double2 a = c.inc[i];
            xd[i] = y;
            a.x = fma(y.x, fq, a.x);
            a.y = fma(y.y, fq, a.y);
            c.inc[i] = a;
          } else {                   // scaled terms b_q = (B b_{q-1}) / q, summed compensated
            y = dw_scale(y, c_dw_inv[q]);
            xd[i] = y;
            DwAcc* a = reinterpret_cast<DwAcc*>(c.inc) + i;
            acc_add4(*a, y);
          }
        }
        team_sync<CLUSTER>();
      }
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        double2 v = c.psi[i];
        double2 a;
        if constexpr (kF64<T>) a = c.inc[i];
        else a = to_d2(reinterpret_cast<const DwAcc*>(c.inc)[i]);
        v.x += a.x;
        v.y += a.y;
        c.psi[i] = v;
      }
    }
    // psi now holds psi_{n+1}
    if (rec) {
      double2* const sg = seg_state(p, n + 1, team) + r0;
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) sg[i] = c.psi[i];
      continue;
    }
    if (p.omega) {
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        const double2 v = c.psi[i];
        c2acc = fma(p.omega[r0 + i], v.x * v.x + v.y * v.y, c2acc);
      }
    }
    if (p.w_tint != 0.0) {   // per-step overlap partial for C3 (App. A)
      double2 gl = make_double2(0.0, 0.0);
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) cmac_conj(gl, p.target[col0 + i], c.psi[i]);
      const double gx = block_sum(gl.x, red);
      const double gy = block_sum(gl.y, red);
      if (threadIdx.x == 0) p.part_g3[(int64_t)part * p.N + n] = make_double2(gx, gy);
    }
    if (p.ckpt_every > 0 && (n + 1) % p.ckpt_every == 0) {
      const int slot = (n + 1) / p.ckpt_every - 1;
      if (slot < p.n_ckpt) {
        double2* dst = p.ckpt + ((int64_t)slot * p.n_states + team) * p.dim + r0;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) dst[i] = c.psi[i];
      }
    }
  }
  if (!rec) {
    double2 gl = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const double2 v = c.psi[i];
      p.psiN[col0 + i] = v;
      cmac_conj(gl, p.target[col0 + i], v);
    }
    const double gx = block_sum(gl.x, red);
    const double gy = block_sum(gl.y, red);
    const double c2 = block_sum(c2acc, red);
    if (threadIdx.x == 0) {
      p.part_g[part] = make_double2(gx, gy);
      p.part_c2[part] = c2;
    }
  }
  team_sync<CLUSTER>();   // no CTA leaves while a team member may still read its shared memory
}

template <typename T, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) k_forward(const __grid_constant__ SweepParams p) {
  forward_body<T, CLUSTER>(p, blockIdx.x);
}

// ------------------------------------------------------------------ backward sweep: shared pieces
//
// For every step n = N..1 and substep l = s-1..0 (B = -i dt H_n / s, P = e^B_m):
//   phase A  psi^(l) = P(-B) psi^(l+1) (adjoint re-propagation, Fig. 1(b)) and the Horner chain
//            w_{m-1} = chi/m!,  w_p = chi/(p+1)! + (-B) w_{p+1},  chi^(l) = w_{-1} = P(-B) chi^(l+1)
//   phase B  x_0 = psi^(l), x_{p+1} = B x_p, and W_ij += conj(w_p[i]) x_p[j] on control entries
// so that  sum_l <chi^(l+1)| dP/du_k |psi^(l)> = sum_ij (C_k)_ij W_ij with C_k = -i dt h_k / s,
// which is the derivative of the approximant (e^B_m)^s at frozen (m, s) (Eq. (auxiliary equation)):
// dP = sum_q 1/q! sum_{r+p=q-1} B^r C B^p  regrouped as  sum_p <w_p| C |x_p>.
// chi is the combined costate of C1 and C2 (Eqs. (stgradient), (gategradient), (C2stgrad)):
//   chi_N = -(w_fid g / n^2) phi_T + (w_forbid/(N n)) Omega psi_N,
//   chi_{n-1} = U_n^+ chi_n + (w_forbid/(N n)) Omega psi_{n-1}   (n-1 >= 1).

// psi_N and chi_N on the CTA's rows.
__device__ __forceinline__ void costate_init(const SweepParams& p, double2* psi, double2* chi, int64_t col0, int r0,
                                             int nrows, double c2w) {
  const double nS = (double)p.n_states;
  const double2 g = *p.g_final;
  double2 coefA = make_double2(-p.w_fid * g.x / (nS * nS), -p.w_fid * g.y / (nS * nS));
  if (p.w_tint != 0.0) {   // C3 source of the last state: -(w_tint / (N n^2)) g_N phi_T
    const double c3w = -p.w_tint / ((double)p.N * nS * nS);
    const double2 gN = p.g3[p.N - 1];
    coefA.x = fma(c3w, gN.x, coefA.x);
    coefA.y = fma(c3w, gN.y, coefA.y);
  }
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    const double2 v = p.psiN[col0 + i];
    psi[i] = v;
    double2 ch = cmul(coefA, p.target[col0 + i]);
    if (c2w != 0.0) {
      const double w = c2w * p.omega[r0 + i];
      ch.x = fma(w, v.x, ch.x);
      ch.y = fma(w, v.y, ch.y);
    }
    chi[i] = ch;
  }
}

// Phase A of one substep.  wout(p, i, w) stores the Horner vector of index p of local row i.  The
// psi chain psi^(l) = P(-B) psi^(l+1) keeps its FP64 terms unscaled (B^q psi^(l+1)) and sums them
// with the weights (-1)^q / q!; compensated FP32 terms are scaled by -1/q at every step.  FP64
// stores w_p; the compensated bulk runs the scaled recursion w'_{m-1} = chi,
// w'_p = chi - (B w'_{p+1}) / (p+2), w'_p = (p+1)! w_p (magnitudes stay near |chi| instead of
// falling like 1/p!), and stores h_p = w'_p / (p+1), which pairs with the scaled x chain
// b_p = B^p psi / p! exactly as w_p pairs with B^p psi: conj(w_p) B^p psi = conj(h_p) b_p.
template <typename T, bool CLUSTER, typename WOut>
__device__ __forceinline__ void phase_a(Team<T, CLUSTER>& tm, int m, WOut wout) {
  using C2 = cx<T>;
  const Carve<T>& c = tm.c;
  const double fm = c_inv_fact[m];
  for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x) {
    tm.X(0)[i] = from_d2<T>(c.psi[i]);
    c.inc[i] = make_double2(0.0, 0.0);
    if constexpr (kF64<T>) {
      const C2 w0 = from_d2<T>(cscale(c.chi[i], fm));
      tm.X(2)[i] = w0;
      wout(m - 1, i, w0);
    } else {
      const C2 w0 = from_d2<T>(c.chi[i]);
      tm.X(2)[i] = w0;
      wout(m - 1, i, dw_scale(w0, c_dw_inv[m]));
    }
  }
  if constexpr (kF64<T>) {
    if (tm.one_row) {
      // Split cluster barrier.  Term q: the first l1 local entries of the row (reading this CTA's
      // rows of X_{q-1}) before wait(q-1), the other entries after it; X_q is written, the barrier
      // is opened (arrive(q)), and the row's bookkeeping (increment, Horner slot, costate) runs
      // while the other CTAs finish.  X_q goes to buffer q & 1, which the others last read as
      // X_{q-2} before they arrived at barrier q-1.  The loop trip counts are those of a single
      // row loop (l1 is uniform in the warp), so no FP64 instruction is added.
      __syncthreads();
      split_arrive<CLUSTER>();
      const int i = threadIdx.x;
      const bool act = i < tm.nrows;
      const int nleft = tm.la - tm.ea, nrest = (tm.eb - tm.ea) - tm.l1;
      for (int q = 1; q <= m; ++q) {
        const int src = (q - 1) & 1, dst = q & 1;
        const C2* xa = tm.X(src);
        const C2* xw = tm.X(2 + src);
        C2 ya = czero<C2>(), yw = czero<C2>(), w = czero<C2>();
        double2 ch = make_double2(0.0, 0.0);
        if (act) {
          if (tm.ed >= 0) {
            const double b = c.vals[tm.ed].y;
            ya = diag_mul(b, xa[i]);
            yw = diag_mul(b, xw[i]);
          }
          for (int k = 0; k < tm.l1; ++k) {
            const int e = tm.la + k;
            const uint32_t loc = c.lcol[e] & kLocalMask;
            const C2 v = c.vals[e];
            cmacT(ya, v, xa[loc]);
            cmacT(yw, v, xw[loc]);
          }
        }
        split_wait<CLUSTER>();
        if (act) {
          for (int e = tm.c0; e < tm.ci; ++e) {
            const uint32_t enc = c.lcol[e];
            const double b = c.vals[e].y;
            mac_imag(ya, b, xload<T, CLUSTER>(xa, tm.tab[src], enc));
            mac_imag(yw, b, xload<T, CLUSTER>(xw, tm.tab[2 + src], enc));
          }
          for (int e = tm.ci; e < tm.ea; ++e) {
            const uint32_t enc = c.lcol[e];
            const double b = c.vals[e].x;
            mac_real(ya, b, xload<T, CLUSTER>(xa, tm.tab[src], enc));
            mac_real(yw, b, xload<T, CLUSTER>(xw, tm.tab[2 + src], enc));
          }
          for (int k = 0; k < nrest; ++k) {
            const int e = k < nleft ? tm.ea + k : tm.la + tm.l1 + (k - nleft);
            const uint32_t enc = c.lcol[e];
            const C2 v = c.vals[e];
            cmacT(ya, v, xload<T, CLUSTER>(xa, tm.tab[src], enc));
            cmacT(yw, v, xload<T, CLUSTER>(xw, tm.tab[2 + src], enc));
          }
          tm.X(dst)[i] = ya;   // B^q psi^(l+1), unscaled
          ch = c.chi[i];
          if (q < m) {
            w = horner(ch, c_inv_fact[m - q], yw);
            tm.X(2 + dst)[i] = w;
          }
        }
        __syncthreads();
        split_arrive<CLUSTER>();
        if (act) {
          double2 a = c.inc[i];
          const double sq = c_sgn_fact[q];   // (-B)^q / q! = (-1)^q / q! B^q
          a.x = fma(ya.x, sq, a.x);
          a.y = fma(ya.y, sq, a.y);
          c.inc[i] = a;
          const double fq = c_inv_fact[m - q];
          if (q < m)
            wout(m - 1 - q, i, w);
          else
            c.chi[i] = make_double2(fma(ch.x, fq, -yw.x), fma(ch.y, fq, -yw.y));
        }
      }
      split_wait<CLUSTER>();
      for (int j = threadIdx.x; j < tm.nrows; j += blockDim.x) {
        double2 v = c.psi[j];
        const double2 a = c.inc[j];
        v.x += a.x;
        v.y += a.y;
        c.psi[j] = v;
      }
      return;
    }
  }
  team_sync<CLUSTER>();
  for (int q = 1; q <= m; ++q) {
    const int src = (q - 1) & 1, dst = q & 1;
    const double fq = c_inv_fact[m - q];
    for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x) {
      C2 ya, yw;
      row_mv2<T, CLUSTER>(c.vals, c.lcol, c.lrow[i], c.lrow[i + 1], tm.X(src), tm.tab[src], tm.X(2 + src),
                          tm.tab[2 + src], ya, yw);
      const double2 ch = c.chi[i];
      if constexpr (kF64<T>) {                       // FP64: B^q psi unscaled, the sum takes (-1)^q / q!
        double2 a = c.inc[i];
        tm.X(dst)[i] = ya;
        const double sq = c_sgn_fact[q];
        a.x = fma(ya.x, sq, a.x);
        a.y = fma(ya.y, sq, a.y);
        c.inc[i] = a;
        if (q < m) {
          const C2 w = horner(ch, fq, yw);           // chi/(p+1)! + (-B) w_{p+1}
          tm.X(2 + dst)[i] = w;
          wout(m - 1 - q, i, w);
        } else {
          c.chi[i] = make_double2(fma(ch.x, fq, -yw.x), fma(ch.y, fq, -yw.y));   // chi^(l) = w_{-1}
        }
      } else {
        ya = dw_scale(ya, c_dw_inv[q]);              // a_q = ((-B) a_{q-1}) / q
        ya = make_float4(-ya.x, -ya.y, -ya.z, -ya.w);
        tm.X(dst)[i] = ya;
        acc_add4(reinterpret_cast<DwAcc*>(c.inc)[i], ya);
        if (q < m) {                                 // w'_p = chi - (B w'_{p+1}) / (p+2), p = m-1-q
          const C2 w = dw_sub(from_d2<T>(ch), dw_scale(yw, c_dw_inv[m - q + 1]));
          tm.X(2 + dst)[i] = w;
          wout(m - 1 - q, i, dw_scale(w, c_dw_inv[m - q]));
        } else {
          const double2 yd = to_d2(yw);              // chi^(l) = w'_{-1} = chi - B w'_0
          c.chi[i] = make_double2(ch.x - yd.x, ch.y - yd.y);
        }
      }
    }
    team_sync<CLUSTER>();
  }
  for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x) {
    double2 v = c.psi[i];
    double2 a;
    if constexpr (kF64<T>) a = c.inc[i];
    else a = to_d2(reinterpret_cast<const DwAcc*>(c.inc)[i]);
    v.x += a.x;
    v.y += a.y;
    c.psi[i] = v;                                  // psi^(l)
  }
}

// Phase B of one substep.  X[4] must hold psi^(l) (own rows) on entry; win(p, i) returns the Horner
// vector of index p of row i (w_p, or h_p for the compensated bulk, whose x chain is scaled:
// b_{p+1} = (B b_p) / (p+1)).
template <typename T, bool CLUSTER, typename WIn>
__device__ __forceinline__ void phase_b(Team<T, CLUSTER>& tm, int m, WIn win) {
  using C2 = cx<T>;
  constexpr bool kStage = !kF64<T>;             // compensated bulk: stage W per substep
  const Carve<T>& c = tm.c;
  // With one row per thread, w_{p+1} is fetched while term p runs (it may come from L2).
  const bool one_row = tm.nrows <= (int)blockDim.x;
  if constexpr (kF64<T>) {
    if (tm.one_row) {
      // Split cluster barrier as in phase A: the first l1 local entries before the wait, the rest
      // after it.  The last term writes nothing that others read, so it ends after its wait.
      __syncthreads();
      split_arrive<CLUSTER>();
      const int i = threadIdx.x;
      const bool act = i < tm.nrows;
      const int nleft = tm.la - tm.ea, nrest = (tm.eb - tm.ea) - tm.l1;
      C2 wnext = act ? win(0, i) : czero<C2>();
      for (int pp = 0; pp < m; ++pp) {
        const int src = pp & 1, dst = src ^ 1;
        const bool more = pp < m - 1;
        const C2* xs = tm.X(4 + src);
        C2 wp = wnext, y0 = czero<C2>();
        auto entry = [&](int e, const C2 x, uint32_t enc) {
          if (more) cmacT(y0, c.vals[e], x);
          if (enc & kCtrlBit) {
            double2 acc = c.W[e];
            cmac_conjT(acc, wp, x);
            c.W[e] = acc;
          }
        };
        if (act) {
          if (more) wnext = win(pp + 1, i);
          if (tm.ed >= 0) {
            const C2 x = xs[i];
            if (more) y0 = diag_mul(c.vals[tm.ed].y, x);
            if (c.lcol[tm.ed] & kCtrlBit) {
              double2 acc = c.W[tm.ed];
              cmac_conjT(acc, wp, x);
              c.W[tm.ed] = acc;
            }
          }
          for (int k = 0; k < tm.l1; ++k) {
            const int e = tm.la + k;
            const uint32_t enc = c.lcol[e];
            entry(e, xs[enc & kLocalMask], enc);
          }
        }
        split_wait<CLUSTER>();
        if (act) {
          // single-phase entries: two multiplies for the chain (imaginary B_ij, then real B_ij)
          auto single = [&](int e, bool imag) {
            const uint32_t enc = c.lcol[e];
            const C2 x = xload<T, CLUSTER>(xs, tm.tab[4 + src], enc);
            if (more) {
              if (imag)
                mac_imag(y0, c.vals[e].y, x);
              else
                mac_real(y0, c.vals[e].x, x);
            }
            if (enc & kCtrlBit) {
              double2 acc = c.W[e];
              cmac_conjT(acc, wp, x);
              c.W[e] = acc;
            }
          };
          for (int e = tm.c0; e < tm.ci; ++e) single(e, true);
          for (int e = tm.ci; e < tm.ea; ++e) single(e, false);
          for (int k = 0; k < nrest; ++k) {
            const int e = k < nleft ? tm.ea + k : tm.la + tm.l1 + (k - nleft);
            const uint32_t enc = c.lcol[e];
            entry(e, xload<T, CLUSTER>(xs, tm.tab[4 + src], enc), enc);
          }
          if (more) tm.X(4 + dst)[i] = y0;
        }
        if (more) {
          __syncthreads();
          split_arrive<CLUSTER>();
        }
      }
      return;
    }
  }
  C2 wnext = (one_row && (int)threadIdx.x < tm.nrows) ? win(0, threadIdx.x) : czero<C2>();
  team_sync<CLUSTER>();
  for (int pp = 0; pp < m; ++pp) {
    const int src = pp & 1, dst = src ^ 1;
    const bool more = pp < m - 1;
    const C2* xs = tm.X(4 + src);
    for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x) {
      C2 wp;
      if (one_row) {
        wp = wnext;
        if (more) wnext = win(pp + 1, i);
      } else {
        wp = win(pp, i);
      }
      const int ea = c.lrow[i], eb = c.lrow[i + 1];
      if constexpr (kF64<T>) {   // FP64: one accumulator, exact loop
        C2 y0 = czero<C2>();
        for (int e = ea; e < eb; ++e) {
          const uint32_t enc = c.lcol[e];
          const C2 x = xload<T, CLUSTER>(xs, tm.tab[4 + src], enc);
          if (more) cmacT(y0, c.vals[e], x);
          if (enc & kCtrlBit) {
            double2 acc = c.W[e];
            cmac_conjT(acc, wp, x);
            c.W[e] = acc;
          }
        }
        if (more) tm.X(4 + dst)[i] = y0;
      } else {
        DwAcc y0 = acc_zero(), y1 = acc_zero();
        int e = ea;
        for (; e + 2 <= eb; e += 2) {
          const uint32_t c0 = c.lcol[e], c1 = c.lcol[e + 1];
          const C2 x0 = xload<T, CLUSTER>(xs, tm.tab[4 + src], c0);
          const C2 x1 = xload<T, CLUSTER>(xs, tm.tab[4 + src], c1);
          if (more) {
            cmacT(y0, c.vals[e], x0);
            cmacT(y1, c.vals[e + 1], x1);
          }
          if (c0 & kCtrlBit) cmac_conjT(c.Wb[e], wp, x0);
          if (c1 & kCtrlBit) cmac_conjT(c.Wb[e + 1], wp, x1);
        }
        if (e < eb) {
          const uint32_t c0 = c.lcol[e];
          const C2 x0 = xload<T, CLUSTER>(xs, tm.tab[4 + src], c0);
          if (more) cmacT(y0, c.vals[e], x0);
          if (c0 & kCtrlBit) cmac_conjT(c.Wb[e], wp, x0);
        }
        if (more) {
          acc_add(y0.sr, y0.cr, y1.sr, y1.cr);
          acc_add(y0.si, y0.ci, y1.si, y1.ci);
          tm.X(4 + dst)[i] = dw_scale(dw_norm(y0), c_dw_inv[pp + 1]);
        }
      }
    }
    if (more) team_sync<CLUSTER>();
  }
  if constexpr (kStage) {   // fold the substep's compensated sums into the FP64 accumulators (row owner)
    for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x)
      for (int e = c.lrow[i]; e < c.lrow[i + 1]; ++e)
        if (c.lcol[e] & kCtrlBit) {
          const double2 b = to_d2(c.Wb[e]);
          double2 a = c.W[e];
          a.x += b.x;
          a.y += b.y;
          c.W[e] = a;
          c.Wb[e] = acc_zero();
        }
  }
}

__device__ __forceinline__ void zero_w(const SweepParams& p, double2* W, DwAcc* Wb, int nnz_loc, bool staged) {
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) {
    W[e] = make_double2(0.0, 0.0);
    if (staged) Wb[e] = acc_zero();
  }
}

// Step end on the psi/chi side: checkpoint reset of psi_{n} and the C2 source of chi.
__device__ __forceinline__ void step_end(const SweepParams& p, double2* psi, double2* chi, int n, int col, int r0,
                                         int nrows, double c2w) {
  if (n <= 0) return;
  if (p.w_tint != 0.0) {   // C3 source: -(w_tint / (N n^2)) g_n phi_T for the state psi_n (App. A recursion)
    const double nS = (double)p.n_states;
    const double c3w = -p.w_tint / ((double)p.N * nS * nS);
    const double2 gn = p.g3[n - 1];
    const double2 cf = make_double2(c3w * gn.x, c3w * gn.y);
    const double2* tg = p.target + (int64_t)col * p.dim + r0;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const double2 t = tg[i];
      double2 ch = chi[i];
      ch.x += cf.x * t.x - cf.y * t.y;
      ch.y += cf.x * t.y + cf.y * t.x;
      chi[i] = ch;
    }
  }
  if (p.ckpt_every > 0 && n % p.ckpt_every == 0 && n / p.ckpt_every - 1 < p.n_ckpt) {
    const double2* srcp = p.ckpt + ((int64_t)(n / p.ckpt_every - 1) * p.n_states + col) * p.dim + r0;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) psi[i] = srcp[i];
  }
  if (c2w != 0.0) {
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      const double w = c2w * p.omega[r0 + i];
      const double2 v = psi[i];
      double2 ch = chi[i];
      ch.x = fma(w, v.x, ch.x);
      ch.y = fma(w, v.y, ch.y);
      chi[i] = ch;
    }
  }
}

// dC/du_kn part = 2 Re sum_ij (C_k)_ij W_ij, C_k = -i (dt/s) h_k: Re(-i h W) = h.x W.y + h.y W.x
__device__ __forceinline__ void grad_partials(const SweepParams& p, const double2* W, int rank, int out_part, int n,
                                              int s, int64_t e0, double* red) {
  const double gscale = 2.0 * p.dt / s;
  for (int k = 0; k < p.K; ++k) {
    const int lo = p.cslice[(k * p.CL + rank) * 2], hi = p.cslice[(k * p.CL + rank) * 2 + 1];
    double acc = 0.0;
    for (int cc = lo + threadIdx.x; cc < hi; cc += blockDim.x) {
      const int e = (int)(p.cidx[cc] - e0);
      const double2 w = W[e];
      const double2 h = p.cval[cc];
      acc = fma(h.x, w.y, acc);
      acc = fma(h.y, w.x, acc);
    }
    const double tot = block_sum(acc, red);
    if (threadIdx.x == 0) p.part_grad[((int64_t)out_part * p.N + n) * p.K + k] = gscale * tot;
  }
}

template <typename T, bool CLUSTER>
__device__ __forceinline__ void team_init(Team<T, CLUSTER>& tm, unsigned char* smem, XTab<T>* tab, const SweepParams& p,
                                          int part, int rank) {
  tm.rank = rank;
  tm.CL = p.CL;
  tm.R = p.R;
  tm.r0 = min(rank * p.R, p.dim);
  const int r1 = min(tm.r0 + p.R, p.dim);
  tm.nrows = r1 - tm.r0;
  tm.e0 = p.rowptr[tm.r0];
  tm.nnz_loc = (int)(p.rowptr[r1] - tm.e0);
  tm.c = carve<T>(smem, p, true, part);
  tm.tab = tab;
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL)
      for (int b = 0; b < 6; ++b) tab[b].ptr[threadIdx.x] = cl.map_shared_rank(tm.X(b), threadIdx.x);
  }
  sweep_setup(p, tm.c.lrow, tm.c.lcol, tm.r0, tm.nrows, tm.e0, tm.nnz_loc);
  tm.one_row = kF64<T> && tm.nrows <= (int)blockDim.x;
  tm.ea = tm.eb = tm.la = tm.l1 = tm.c0 = tm.ci = 0;
  tm.ed = -1;
  __syncthreads();   // the local pattern
  if (tm.one_row) {
    int nloc = 1 << 30;
    if ((int)threadIdx.x < tm.nrows) {
      const int* lrow = tm.c.lrow;
      const uint32_t* lcol = tm.c.lcol;
      tm.ea = lrow[threadIdx.x];
      tm.eb = lrow[threadIdx.x + 1];
      if (diag_at(p, lcol, tm.ea, tm.eb, rank, threadIdx.x)) tm.ed = tm.ea++;
      tm.c0 = tm.ea;
      row_segments(lcol, tm.c0, tm.eb, &tm.ci, &tm.ea);
      int a = tm.ea;
      while (a < tm.eb && ((lcol[a] >> kOwnerShift) & 0xFFu) < (uint32_t)rank) ++a;
      int b = a;
      while (b < tm.eb && ((lcol[b] >> kOwnerShift) & 0xFFu) == (uint32_t)rank) ++b;
      tm.la = a;
      nloc = b - a;
    }
    const int wmin = __reduce_min_sync(0xffffffffu, nloc);
    tm.l1 = wmin == (1 << 30) ? 0 : wmin;
  }
}

// ------------------------------------------------------------------ backward sweep, one team per column

template <typename T, bool CLUSTER>
__device__ __forceinline__ void backward_body(const SweepParams& p, const int part) {
  using C2 = cx<T>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<T> tab[6];
  const int col = part / p.CL, rank = part % p.CL;
  Team<T, CLUSTER> tm;
  team_init<T, CLUSTER>(tm, smem, tab, p, part, rank);
  const Carve<T>& c = tm.c;
  const int64_t col0 = (int64_t)col * p.dim + tm.r0;
  const double c2w = (p.omega && p.w_forbid != 0.0) ? p.w_forbid / ((double)p.N * p.n_states) : 0.0;
  const int R = p.R, m_smem = p.m_smem;
  costate_init(p, c.psi, c.chi, col0, tm.r0, tm.nrows, c2w);
  team_sync<CLUSTER>();
  auto slot = [&](int pp, int i) -> C2* {
    return pp < m_smem ? c.wsm + (int64_t)pp * R + i : c.wgl + (int64_t)(pp - m_smem) * R + i;
  };
  for (int n = p.N - 1; n >= 0; --n) {
    const int m = p.ms_m[n], s = p.ms_s[n];
    if (s <= 0 || m <= 0) continue;
    load_controls(p, n, s_u);
    __syncthreads();
    assemble<T>(p, c.vals, tm.e0, tm.nnz_loc, p.dt / s, s_u);
    zero_w(p, c.W, c.Wb, tm.nnz_loc, !kF64<T>);
    __syncthreads();
    for (int l = s - 1; l >= 0; --l) {
      phase_a<T, CLUSTER>(tm, m, [&](int pp, int i, C2 w) { *slot(pp, i) = w; });
      for (int i = threadIdx.x; i < tm.nrows; i += blockDim.x) tm.X(4)[i] = from_d2<T>(c.psi[i]);
      phase_b<T, CLUSTER>(tm, m, [&](int pp, int i) -> C2 { return *slot(pp, i); });
    }
    __syncthreads();
    step_end(p, c.psi, c.chi, n, col, tm.r0, tm.nrows, c2w);
    grad_partials(p, c.W, rank, part, n, s, tm.e0, red);
    __syncthreads();
  }
  team_sync<CLUSTER>();
}

template <typename T, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) k_backward(const __grid_constant__ SweepParams p) {
  if (p.gate_on_flag && *p.plan_flag == 0) return;   // the three-stage backward ran (uniform over the grid)
  backward_body<T, CLUSTER>(p, blockIdx.x);
}

// ------------------------------------------------------------------ three-stage backward
//
// The backward sweep split by role.  Its only sequential part is the costate chain: for every step
// n = N..1 and substep l = s-1..0 the Horner recursion
//     w_{m-1} = chi/m!,   w_p = chi/(p+1)! + (-B) w_{p+1},   chi^(l) = w_{-1} = P(-B) chi^(l+1)
// (m products per substep on one team of CL CTAs per column: k_costate), which stores every w_p of a
// block of steps.  The states are not re-propagated backwards: the forward sweep stored psi_n of
// every step, and the Taylor vectors x_p = B^p psi^(l), psi^(l) = P^l psi_n, do not depend on the
// costate, so k_gradient regenerates them for all steps of a block side by side, on the SMs the
// chain leaves idle, and accumulates W_ij += conj(w_p[i]) x_p[j] once the block's w_p are stored.
// This is the fused sweep's derivative (Eq. (auxiliary equation), dP regrouped as
// sum_p <w_p| C |x_p>), evaluated on the forward's own psi^(l).
//
// Launch order per block b (descending): k_costate(b) on the critical stream, then k_gradient(b) on
// a second stream after an event; the block buffers alternate, and k_costate(b - 2) waits for
// k_gradient(b).  No kernel waits for another one on the device.

// psi_n, the input state of step n: from the segment buffer when checkpoints are M > 1 steps apart
// (the segment was recomputed), else psi_0 or the state the forward stored after step n - 1.
__device__ __forceinline__ const double2* step_state(const SweepParams& p, int n, int col) {
  if (p.seg) return seg_state(p, n, col);
  return n == 0 ? p.psi0 + (int64_t)col * p.dim : p.ckpt + ((int64_t)(n - 1) * p.n_states + col) * p.dim;
}

// Terms of the block's steps [n_begin, n): the offset of step n's first Horner vector in the block buffer.
__device__ __forceinline__ int64_t block_term_offset(const SweepParams& p, int n) {
  int64_t t = 0;
  for (int k = p.n_begin; k < n; ++k) {
    const int mk = p.ms_m[k], sk = p.ms_s[k];
    if (mk > 0 && sk > 0) t += (int64_t)mk * sk;
  }
  return t;
}

// One block: does every block of steps fit the Horner buffers?  Sets *flag = 0 (three-stage path)
// or 1 (the fused backward runs).
__global__ void __launch_bounds__(256) k_plan(PlanParams p) {
  __shared__ int over;
  if (threadIdx.x == 0) over = 0;
  __syncthreads();
  const int nb = (p.N + p.steps_per_block - 1) / p.steps_per_block;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    int64_t t = 0;
    const int n1 = min(p.N, (b + 1) * p.steps_per_block);
    for (int n = b * p.steps_per_block; n < n1; ++n) {
      const int m = p.ms_m[n], s = p.ms_s[n];
      if (m > 0 && s > 0) t += (int64_t)m * s;
    }
    if (t > p.cap_terms) over = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) *p.flag = over;
}

// chi_N = -(w_fid g / n^2) phi_T + (w_forbid/(N n)) Omega psi_N (+ the C3 source of psi_N) on the CTA's rows.
__device__ __forceinline__ void costate_final(const SweepParams& p, double2* chi, int64_t col0, int r0, int nrows,
                                              double c2w) {
  const double nS = (double)p.n_states;
  const double2 g = *p.g_final;
  double2 coefA = make_double2(-p.w_fid * g.x / (nS * nS), -p.w_fid * g.y / (nS * nS));
  if (p.w_tint != 0.0) {
    const double c3w = -p.w_tint / ((double)p.N * nS * nS);
    const double2 gN = p.g3[p.N - 1];
    coefA.x = fma(c3w, gN.x, coefA.x);
    coefA.y = fma(c3w, gN.y, coefA.y);
  }
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    double2 ch = cmul(coefA, p.target[col0 + i]);
    if (c2w != 0.0) {
      const double w = c2w * p.omega[r0 + i];
      const double2 v = p.psiN[col0 + i];
      ch.x = fma(w, v.x, ch.x);
      ch.y = fma(w, v.y, ch.y);
    }
    chi[i] = ch;
  }
}

// Costate chain over the block [n_begin, n_end), one team per column (the forward sweep's partition
// and shared-memory layout; its psi rows hold chi here).  chi enters from p.chi_io (or chi_N in the
// last block) and leaves through it.
template <typename T, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) k_costate(SweepParams p) {
  using C2 = cx<T>;
  if (*p.plan_flag != 0) return;   // the fused backward runs instead (the same word for the whole grid)
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<T> tab[2];
  const int part = blockIdx.x;
  const int col = part / p.CL, rank = part % p.CL;
  const int r0 = min(rank * p.R, p.dim), r1 = min(r0 + p.R, p.dim), nrows = r1 - r0;
  const int64_t e0 = p.rowptr[r0];
  const int nnz_loc = (int)(p.rowptr[r1] - e0);
  const Carve<T> c = carve<T>(smem, p, false, part);
  C2* const X0 = c.xb;
  double2* const chi = c.psi;
  const int R = p.R;
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL) {
      tab[0].ptr[threadIdx.x] = cl.map_shared_rank(X0, threadIdx.x);
      tab[1].ptr[threadIdx.x] = cl.map_shared_rank(X0 + R, threadIdx.x);
    }
  }
  sweep_setup(p, c.lrow, c.lcol, r0, nrows, e0, nnz_loc);
  const int64_t col0 = (int64_t)col * p.dim + r0;
  const double c2w = (p.omega && p.w_forbid != 0.0) ? p.w_forbid / ((double)p.N * p.n_states) : 0.0;
  if (p.n_end == p.N)
    costate_final(p, chi, col0, r0, nrows, c2w);
  else
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) chi[i] = p.chi_io[col0 + i];
  const bool split_rows = nrows <= (int)blockDim.x;
  int ea = 0, eb = 0, la = 0, lb = 0, ed = -1, c0 = 0, ci = 0;
  __syncthreads();   // the local pattern written by sweep_setup
  if (split_rows && (int)threadIdx.x < nrows) {
    ea = c.lrow[threadIdx.x];
    eb = c.lrow[threadIdx.x + 1];
    if (diag_at(p, c.lcol, ea, eb, rank, threadIdx.x)) ed = ea++;
    c0 = ea;
    row_segments(c.lcol, c0, eb, &ci, &ea);
    la = ea;
    while (la < eb && ((c.lcol[la] >> kOwnerShift) & 0xFFu) < (uint32_t)rank) ++la;
    lb = la;
    while (lb < eb && ((c.lcol[lb] >> kOwnerShift) & 0xFFu) == (uint32_t)rank) ++lb;
  }
  team_sync<CLUSTER>();
  C2* const hb = reinterpret_cast<C2*>(p.hbuf);
  const int64_t hstride = (int64_t)p.n_states * p.dim;   // bulk elements per stored term
  int64_t toff = block_term_offset(p, p.n_end);
  for (int n = p.n_end - 1; n >= p.n_begin; --n) {
    const int m = p.ms_m[n], s = p.ms_s[n];
    if (s <= 0 || m <= 0) continue;   // flagged by k_schedule; uniform over the team
    toff -= (int64_t)m * s;
    load_controls(p, n, s_u);
    __syncthreads();
    assemble<T>(p, c.vals, e0, nnz_loc, p.dt / s, s_u);
    __syncthreads();
    for (int l = s - 1; l >= 0; --l) {
      C2* const hl = hb + (toff + (int64_t)l * m) * hstride + col0;   // w_p of substep l: hl[p * hstride + i]
      const double fm = c_inv_fact[m];
      if constexpr (kF64<T>) {
        if (split_rows) {
          // Same split cluster barrier as the forward sweep: term q reads w_{m-q} from buffer
          // (q - 1) & 1 and writes w_{m-1-q} to buffer q & 1.  Thread 0 copies each buffer's rows
          // to the Horner block with one bulk asynchronous copy once the term has written it; a
          // buffer is rewritten two terms later, after thread 0 has waited (before its arrive) for
          // all but its latest copy to finish reading.
          const uint32_t rbytes = (uint32_t)nrows * 16u;
          for (int i = threadIdx.x; i < nrows; i += blockDim.x) X0[i] = from_d2<T>(cscale(chi[i], fm));
          async_proxy_fence();
          __syncthreads();
          if (threadIdx.x == 0 && rbytes) bulk_store(hl + (int64_t)(m - 1) * hstride, X0, rbytes);
          split_arrive<CLUSTER>();
          const int i = threadIdx.x;
          for (int q = 1; q <= m; ++q) {
            const int src = (q - 1) & 1, dst = q & 1;
            const C2* xs = X0 + src * R;
            C2 y = czero<C2>();
            if (i < nrows) {
              if (ed >= 0) y = diag_mul(c.vals[ed].y, xs[i]);
              for (int e = la; e < lb; ++e) cmacT(y, c.vals[e], xs[c.lcol[e] & kLocalMask]);
            }
            split_wait<CLUSTER>();
            if (i < nrows) {
              for (int e = c0; e < ci; ++e) mac_imag(y, c.vals[e].y, xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              for (int e = ci; e < ea; ++e) mac_real(y, c.vals[e].x, xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              const int nl = la - ea, nr = nl + (eb - lb);
              for (int k = 0; k < nr; ++k) {
                const int e = k < nl ? ea + k : lb + (k - nl);
                cmacT(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              }
              const double2 ch = chi[i];
              if (q < m) {
                y = horner(ch, c_inv_fact[m - q], y);   // w_{m-1-q} = chi/(m-q)! + (-B) w_{m-q}
                X0[dst * R + i] = y;
              } else {
                chi[i] = make_double2(fma(ch.x, c_inv_fact[0], -y.x), fma(ch.y, c_inv_fact[0], -y.y));   // w_{-1}
              }
            }
            if (q < m) {
              async_proxy_fence();
              __syncthreads();
              if (threadIdx.x == 0 && rbytes) {
                bulk_store(hl + (int64_t)(m - 1 - q) * hstride, X0 + dst * R, rbytes);
                bulk_wait_read<1>();   // the copy of the other buffer has read it
              }
              split_arrive<CLUSTER>();
            } else {
              if (threadIdx.x == 0) bulk_wait_read<0>();   // the next substep rewrites buffer 0
              team_sync<CLUSTER>();
            }
          }
          continue;
        }
      } else {
        if (split_rows) {
          // The compensated bulk's Horner chain with the split cluster barrier: the scaled recursion
          // w'_{m-1} = chi, w'_p = chi - (B w'_{p+1}) / (p+2); the w'_p go to the Horner block by the
          // same bulk copies as in FP64 (k_gradient applies the 1/(p+1)); chi's pair in a register.
          const int i = threadIdx.x;
          const uint32_t rbytes = (uint32_t)nrows * 16u;
          C2 chb = czero<C2>();
          if (i < nrows) {
            chb = from_d2<T>(chi[i]);
            X0[i] = chb;
          }
          async_proxy_fence();
          __syncthreads();
          if (threadIdx.x == 0 && rbytes) bulk_store(hl + (int64_t)(m - 1) * hstride, X0, rbytes);
          split_arrive<CLUSTER>();
          for (int q = 1; q <= m; ++q) {
            const int src = (q - 1) & 1, dst = q & 1;
            const C2* xs = X0 + src * R;
            DwAcc y = acc_zero();
            if (i < nrows) {
              if (ed >= 0) dw_mac_imag(y, c.vals[ed], xs[i]);
              for (int e = la; e < lb; ++e) cmacT(y, c.vals[e], xs[c.lcol[e] & kLocalMask]);
            }
            split_wait<CLUSTER>();
            if (i < nrows) {
              for (int e = c0; e < ci; ++e) dw_mac_imag(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              for (int e = ci; e < ea; ++e) dw_mac_real(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              const int nl = la - ea, nr = nl + (eb - lb);
              for (int k = 0; k < nr; ++k) {
                const int e = k < nl ? ea + k : lb + (k - nl);
                cmacT(y, c.vals[e], xload<T, CLUSTER>(xs, tab[src], c.lcol[e]));
              }
              if (q < m) {
                X0[dst * R + i] = dw_sub(chb, dw_scale(dw_norm(y), c_dw_inv[m - q + 1]));
              } else {
                const double2 yd = to_d2(y);   // chi^(l) = w'_{-1} = chi - B w'_0
                const double2 ch = chi[i];
                chi[i] = make_double2(ch.x - yd.x, ch.y - yd.y);
              }
            }
            if (q < m) {
              async_proxy_fence();
              __syncthreads();
              if (threadIdx.x == 0 && rbytes) {
                bulk_store(hl + (int64_t)(m - 1 - q) * hstride, X0 + dst * R, rbytes);
                bulk_wait_read<1>();
              }
              split_arrive<CLUSTER>();
            } else {
              if (threadIdx.x == 0) bulk_wait_read<0>();
              team_sync<CLUSTER>();
            }
          }
          continue;
        }
      }
      // Generic loop.  The compensated bulk runs the scaled recursion w'_{m-1} = chi,
      // w'_p = chi - (B w'_{p+1}) / (p+2) and stores w'_p (k_gradient pairs w'_p / (p+1) with the
      // scaled x chain, see phase_a); its copy of chi as a pair of floats lives in the (otherwise
      // unused) increment rows.
      C2* const chi_b = reinterpret_cast<C2*>(c.inc);
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        if constexpr (kF64<T>) {
          const C2 w = from_d2<T>(cscale(chi[i], fm));
          X0[i] = w;
          hl[(int64_t)(m - 1) * hstride + i] = w;
        } else {
          const C2 w = from_d2<T>(chi[i]);
          chi_b[i] = w;
          X0[i] = w;
          hl[(int64_t)(m - 1) * hstride + i] = w;
        }
      }
      team_sync<CLUSTER>();
      for (int q = 1; q <= m; ++q) {
        const int src = (q - 1) & 1, dst = q & 1;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          const C2 y = row_mv<T, CLUSTER>(c.vals, c.lcol, c.lrow[i], c.lrow[i + 1], X0 + src * R, tab[src]);
          const double2 ch = chi[i];
          if (q < m) {
            if constexpr (kF64<T>) {
              const C2 w = horner(ch, c_inv_fact[m - q], y);
              X0[dst * R + i] = w;
              hl[(int64_t)(m - 1 - q) * hstride + i] = w;
            } else {
              const C2 w = dw_sub(chi_b[i], dw_scale(y, c_dw_inv[m - q + 1]));
              X0[dst * R + i] = w;
              hl[(int64_t)(m - 1 - q) * hstride + i] = w;
            }
          } else {
            const double2 yd = to_d2(y);
            chi[i] = make_double2(fma(ch.x, c_inv_fact[0], -yd.x), fma(ch.y, c_inv_fact[0], -yd.y));
          }
        }
        team_sync<CLUSTER>();
      }
    }
    // end of step n: the sources of the state psi_n (n >= 1), C3 then C2 (App. A recursions)
    if (n >= 1) {
      if (p.w_tint != 0.0) {
        const double nS = (double)p.n_states;
        const double c3w = -p.w_tint / ((double)p.N * nS * nS);
        const double2 gn = p.g3[n - 1];
        const double2 cf = make_double2(c3w * gn.x, c3w * gn.y);
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          const double2 t = p.target[col0 + i];
          double2 ch = chi[i];
          ch.x += cf.x * t.x - cf.y * t.y;
          ch.y += cf.x * t.y + cf.y * t.x;
          chi[i] = ch;
        }
      }
      if (c2w != 0.0) {
        const double2* st = step_state(p, n, col) + r0;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          const double w = c2w * p.omega[r0 + i];
          const double2 v = st[i];
          double2 ch = chi[i];
          ch.x = fma(w, v.x, ch.x);
          ch.y = fma(w, v.y, ch.y);
          chi[i] = ch;
        }
      }
    }
  }
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) p.chi_io[col0 + i] = chi[i];
  if (threadIdx.x == 0) bulk_wait_all();   // the Horner block is complete before the kernel ends
  team_sync<CLUSTER>();   // no CTA leaves while a team member may still read its shared memory
}

// Gradient terms of the block's steps, one team of CL CTAs per (step, column): psi^(0) = psi_n from
// the forward's stored states; per substep l the x chain x_0 = psi^(l), x_{p+1} = B x_p with
// W_ij += conj(w_p[i]) x_p[j] on the control entries (w_p of substep l from k_costate), and
// psi^(l+1) = sum_{q<=m} x_q / q! for the next substep; then the step's partials
// 2 Re sum_ij (C_k)_ij W_ij, C_k = -i dt h_k / s.  Independent across steps and columns.
template <typename T, bool CLUSTER>
__global__ void __launch_bounds__(512, 1) k_gradient(SweepParams p) {
  using C2 = cx<T>;
  constexpr bool kStage = !kF64<T>;   // compensated bulk: W staged per substep
  if (*p.plan_flag != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<T> tab[2];
  const int part = blockIdx.x;
  const int unit = part / p.CL, rank = part % p.CL;
  const int n = p.n_begin + unit / p.n_states, col = unit % p.n_states;
  const int out_part = col * p.CL + rank;
  const int r0 = min(rank * p.R, p.dim), r1 = min(r0 + p.R, p.dim), nrows = r1 - r0;
  const int64_t e0 = p.rowptr[r0];
  const int nnz_loc = (int)(p.rowptr[r1] - e0);
  const SmemLayout L = make_glayout(p.R, p.max_nnz_loc, p.in_smem, (int)sizeof(C2), kStage);
  double2* const scr = p.scratch + (int64_t)part * p.scratch_stride;
  C2* const X0 = reinterpret_cast<C2*>(smem + L.xbuf);
  double2* const psi = reinterpret_cast<double2*>(smem + L.psi);
  double2* const inc = reinterpret_cast<double2*>(smem + L.inc);
  C2* const vals = L.vals >= 0 ? reinterpret_cast<C2*>(smem + L.vals) : reinterpret_cast<C2*>(scr + p.scr_vals);
  double2* const W = L.W >= 0 ? reinterpret_cast<double2*>(smem + L.W) : scr + p.scr_W;
  DwAcc* const Wb = L.Wb >= 0 ? reinterpret_cast<DwAcc*>(smem + L.Wb) : reinterpret_cast<DwAcc*>(scr + p.scr_Wb);
  int* const lrow = reinterpret_cast<int*>(smem + L.lrow);
  uint32_t* const lcol = reinterpret_cast<uint32_t*>(smem + L.lcol);
  const int R = p.R;
  const int m = p.ms_m[n], s = p.ms_s[n];
  if (m <= 0 || s <= 0) {   // flagged by k_schedule (the call returns an error); keep the partials defined
    if (threadIdx.x < p.K) p.part_grad[((int64_t)out_part * p.N + n) * p.K + threadIdx.x] = 0.0;
    return;   // uniform over the team: no team member waits at a barrier or reads this CTA's memory
  }
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL) {
      tab[0].ptr[threadIdx.x] = cl.map_shared_rank(X0, threadIdx.x);
      tab[1].ptr[threadIdx.x] = cl.map_shared_rank(X0 + R, threadIdx.x);
    }
  }
  sweep_setup(p, lrow, lcol, r0, nrows, e0, nnz_loc);
  load_controls(p, n, s_u);
  const double2* st = step_state(p, n, col) + r0;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) psi[i] = st[i];
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) {
    W[e] = make_double2(0.0, 0.0);
    if (kStage) Wb[e] = acc_zero();
  }
  __syncthreads();
  assemble<T>(p, vals, e0, nnz_loc, p.dt / s, s_u);
  const bool one_row = kF64<T> && nrows <= (int)blockDim.x;
  int ea = 0, eb = 0, la = 0, l1 = 0, ed = -1, c0 = 0, ci = 0;
  {
    int nloc = 1 << 30;
    if (one_row && (int)threadIdx.x < nrows) {
      ea = lrow[threadIdx.x];
      eb = lrow[threadIdx.x + 1];
      if (diag_at(p, lcol, ea, eb, rank, threadIdx.x)) ed = ea++;
      c0 = ea;
      row_segments(lcol, c0, eb, &ci, &ea);
      int a = ea;
      while (a < eb && ((lcol[a] >> kOwnerShift) & 0xFFu) < (uint32_t)rank) ++a;
      int b = a;
      while (b < eb && ((lcol[b] >> kOwnerShift) & 0xFFu) == (uint32_t)rank) ++b;
      la = a;
      nloc = b - a;
    }
    const int wmin = __reduce_min_sync(0xffffffffu, nloc);
    l1 = wmin == (1 << 30) ? 0 : wmin;
  }
  const C2* const hb = reinterpret_cast<const C2*>(p.hbuf);
  const int64_t hstride = (int64_t)p.n_states * p.dim;
  const int64_t toff = block_term_offset(p, n);
  __syncthreads();   // vals and the row segments
  for (int l = 0; l < s; ++l) {
    const C2* const hl = hb + (toff + (int64_t)l * m) * hstride + (int64_t)col * p.dim + r0;
    const bool last = l == s - 1;
    for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
      X0[i] = from_d2<T>(psi[i]);
      inc[i] = make_double2(0.0, 0.0);
    }
    bool split_done = false;
    if constexpr (kF64<T>) {
     if (one_row) {
      split_done = true;
      // Split cluster barrier (as in the fused sweep's phase B): term p sums the first l1 local
      // entries before the wait, the rest after it; x_{p+1} goes to buffer (p + 1) & 1.  The last
      // term of the substep ends with a full barrier: the next substep overwrites buffer 0.
      __syncthreads();
      split_arrive<CLUSTER>();
      const int i = threadIdx.x;
      const bool act = i < nrows;
      const int nleft = la - ea, nrest = (eb - ea) - l1;
      C2 wnext = act ? __ldcg(hl + i) : czero<C2>();
      for (int pp = 0; pp < m; ++pp) {
        const int src = pp & 1, dst = src ^ 1;
        const bool more = pp < m - 1 || !last;
        const C2* xs = X0 + src * R;
        const C2 wp = wnext;
        C2 y0 = czero<C2>();
        auto wacc = [&](int e, const C2 x) {
          double2 acc = W[e];
          cmac_conjT(acc, wp, x);
          W[e] = acc;
        };
        if (act) {
          if (pp + 1 < m) wnext = __ldcg(hl + (int64_t)(pp + 1) * hstride + i);
          if (ed >= 0) {
            const C2 x = xs[i];
            if (more) y0 = diag_mul(vals[ed].y, x);
            if (lcol[ed] & kCtrlBit) wacc(ed, x);
          }
          for (int k = 0; k < l1; ++k) {
            const int e = la + k;
            const uint32_t enc = lcol[e];
            const C2 x = xs[enc & kLocalMask];
            if (more) cmacT(y0, vals[e], x);
            if (enc & kCtrlBit) wacc(e, x);
          }
        }
        split_wait<CLUSTER>();
        if (act) {
          for (int e = c0; e < ci; ++e) {
            const uint32_t enc = lcol[e];
            const C2 x = xload<T, CLUSTER>(xs, tab[src], enc);
            if (more) mac_imag(y0, vals[e].y, x);
            if (enc & kCtrlBit) wacc(e, x);
          }
          for (int e = ci; e < ea; ++e) {
            const uint32_t enc = lcol[e];
            const C2 x = xload<T, CLUSTER>(xs, tab[src], enc);
            if (more) mac_real(y0, vals[e].x, x);
            if (enc & kCtrlBit) wacc(e, x);
          }
          for (int k = 0; k < nrest; ++k) {
            const int e = k < nleft ? ea + k : la + l1 + (k - nleft);
            const uint32_t enc = lcol[e];
            const C2 x = xload<T, CLUSTER>(xs, tab[src], enc);
            if (more) cmacT(y0, vals[e], x);
            if (enc & kCtrlBit) wacc(e, x);
          }
          if (more) {
            if (pp < m - 1) X0[dst * R + i] = y0;   // x_{p+1} = B^{p+1} psi^(l), unscaled
            double2 a = inc[i];
            const double f = c_inv_fact[pp + 1];
            a.x = fma(y0.x, f, a.x);
            a.y = fma(y0.y, f, a.y);
            inc[i] = a;
          }
        }
        if (pp < m - 1) {
          __syncthreads();
          split_arrive<CLUSTER>();
        } else {
          team_sync<CLUSTER>();
        }
      }
     }
    }
    if (!split_done) {
      team_sync<CLUSTER>();
      for (int pp = 0; pp < m; ++pp) {
        const int src = pp & 1, dst = src ^ 1;
        const bool more = pp < m - 1 || !last;
        const C2* xs = X0 + src * R;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          C2 wp = __ldcg(hl + (int64_t)pp * hstride + i);
          if constexpr (!kF64<T>) wp = dw_scale(wp, c_dw_inv[pp + 1]);   // h_p = w'_p / (p+1)
          const int ra = lrow[i], rb = lrow[i + 1];
          if constexpr (kF64<T>) {
            C2 y0 = czero<C2>(), y1 = czero<C2>();
            auto wacc = [&](int e, const C2 x) {
              double2 acc = W[e];
              cmac_conjT(acc, wp, x);
              W[e] = acc;
            };
            int e = ra;
            for (; e + 2 <= rb; e += 2) {
              const uint32_t q0 = lcol[e], q1 = lcol[e + 1];
              const C2 x0 = xload<T, CLUSTER>(xs, tab[src], q0);
              const C2 x1 = xload<T, CLUSTER>(xs, tab[src], q1);
              if (more) {
                cmacT(y0, vals[e], x0);
                cmacT(y1, vals[e + 1], x1);
              }
              if (q0 & kCtrlBit) wacc(e, x0);
              if (q1 & kCtrlBit) wacc(e + 1, x1);
            }
            if (e < rb) {
              const uint32_t q0 = lcol[e];
              const C2 x0 = xload<T, CLUSTER>(xs, tab[src], q0);
              if (more) cmacT(y0, vals[e], x0);
              if (q0 & kCtrlBit) wacc(e, x0);
            }
            if (more) {
              const C2 y = make_double2(y0.x + y1.x, y0.y + y1.y);
              if (pp < m - 1) X0[dst * R + i] = y;
              double2 a = inc[i];
              const double f = c_inv_fact[pp + 1];
              a.x = fma(y.x, f, a.x);
              a.y = fma(y.y, f, a.y);
              inc[i] = a;
            }
          } else {   // scaled x chain b_{p+1} = (B b_p) / (p+1), W += conj(h_p) b_p compensated
            DwAcc y0 = acc_zero(), y1 = acc_zero();
            int e = ra;
            for (; e + 2 <= rb; e += 2) {
              const uint32_t q0 = lcol[e], q1 = lcol[e + 1];
              const C2 x0 = xload<T, CLUSTER>(xs, tab[src], q0);
              const C2 x1 = xload<T, CLUSTER>(xs, tab[src], q1);
              if (more) {
                cmacT(y0, vals[e], x0);
                cmacT(y1, vals[e + 1], x1);
              }
              if (q0 & kCtrlBit) cmac_conjT(Wb[e], wp, x0);
              if (q1 & kCtrlBit) cmac_conjT(Wb[e + 1], wp, x1);
            }
            if (e < rb) {
              const uint32_t q0 = lcol[e];
              const C2 x0 = xload<T, CLUSTER>(xs, tab[src], q0);
              if (more) cmacT(y0, vals[e], x0);
              if (q0 & kCtrlBit) cmac_conjT(Wb[e], wp, x0);
            }
            if (more) {
              acc_add(y0.sr, y0.cr, y1.sr, y1.cr);
              acc_add(y0.si, y0.ci, y1.si, y1.ci);
              const C2 y = dw_scale(dw_norm(y0), c_dw_inv[pp + 1]);
              if (pp < m - 1) X0[dst * R + i] = y;
              acc_add4(reinterpret_cast<DwAcc*>(inc)[i], y);
            }
          }
        }
        team_sync<CLUSTER>();
      }
      if constexpr (kStage) {   // fold the substep's compensated sums into the FP64 accumulators (row owner)
        for (int i = threadIdx.x; i < nrows; i += blockDim.x)
          for (int e = lrow[i]; e < lrow[i + 1]; ++e)
            if (lcol[e] & kCtrlBit) {
              const double2 b = to_d2(Wb[e]);
              double2 a = W[e];
              a.x += b.x;
              a.y += b.y;
              W[e] = a;
              Wb[e] = acc_zero();
            }
      }
    }
    if (!last)
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        double2 v = psi[i];
        double2 a;
        if constexpr (kF64<T>) a = inc[i];
        else a = to_d2(reinterpret_cast<const DwAcc*>(inc)[i]);
        v.x += a.x;
        v.y += a.y;
        psi[i] = v;   // psi^(l+1)
      }
  }
  __syncthreads();
  grad_partials(p, W, rank, out_part, n, s, e0, red);
  team_sync<CLUSTER>();   // no CTA leaves while a team member may still read its shared memory
}

// ------------------------------------------------------------------ finalize (one block)

// The partials are read through L2 (__ldcg): in the batch work queue they were written by other
// CTAs of the same launch, whose writes this SM's L1 need not hold.
__device__ __forceinline__ void finalize_body(const FinalizeParams& p) {
  __shared__ double red[32];
  double gx = 0.0, gy = 0.0, c2 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < p.n_parts; i += blockDim.x) {
    const double2 g = __ldcg(p.part_g + i);
    gx += g.x;
    gy += g.y;
    c2 += __ldcg(p.part_c2 + i);
  }
  for (int64_t i = threadIdx.x; i < (int64_t)p.K * p.N; i += blockDim.x) a2 = fma(p.u[i], p.u[i], a2);
  double g3sq = 0.0;
  if (p.part_g3) {   // per-step overlaps g_n (C3): fixed-order sums over the partials
    for (int n = threadIdx.x; n < p.N; n += blockDim.x) {
      double sx = 0.0, sy = 0.0;
      for (int i = 0; i < p.n_parts; ++i) {
        const double2 v = __ldcg(p.part_g3 + (int64_t)i * p.N + n);
        sx += v.x;
        sy += v.y;
      }
      p.g3_out[n] = make_double2(sx, sy);
      g3sq = fma(sx, sx, fma(sy, sy, g3sq));
    }
  }
  gx = block_sum(gx, red);
  gy = block_sum(gy, red);
  c2 = block_sum(c2, red);
  a2 = block_sum(a2, red);
  g3sq = block_sum(g3sq, red);
  if (threadIdx.x == 0) {
    const double n = (double)p.n_states;
    const double C1 = 1.0 - (gx * gx + gy * gy) / (n * n);
    const double C2 = c2 / ((double)p.N * n);
    const double Ca = a2 / (double)p.N;
    const double C3 = p.part_g3 ? 1.0 - g3sq / ((double)p.N * n * n) : 0.0;
    *p.g_out = make_double2(gx, gy);
    *p.cost_out = p.w_fid * C1 + p.w_forbid * C2 + p.w_amp * Ca + (p.part_g3 ? p.w_tint * C3 : 0.0);
    if (p.parts_out) {
      p.parts_out[0] = C1;
      p.parts_out[1] = C2;
      p.parts_out[2] = Ca;
      p.parts_out[3] = sqrt(gx * gx + gy * gy);
      p.parts_out[4] = C3;
    }
  }
}

__global__ void __launch_bounds__(256) k_finalize(const __grid_constant__ FinalizeParams p) { finalize_body(p); }

// ------------------------------------------------------------------ gradient reduce

__device__ __forceinline__ void grad_reduce_body(const GradReduceParams& p, const int64_t first, const int64_t stride) {
  const int64_t total = (int64_t)p.K * p.N;
  for (int64_t idx = first; idx < total; idx += stride) {
    const int k = (int)(idx / p.N), n = (int)(idx % p.N);
    const int n_parts = (p.plan_flag && *p.plan_flag != 0) ? p.n_parts_alt : p.n_parts;
    double acc = 0.0;
    for (int part = 0; part < n_parts; ++part) acc += __ldcg(p.part_grad + ((int64_t)part * p.N + n) * p.K + k);
    p.grad[idx] = acc + p.w_amp * 2.0 * p.u[idx] / (double)p.N;
  }
}

__global__ void k_grad_reduce(const __grid_constant__ GradReduceParams p) {
  grad_reduce_body(p, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// ------------------------------------------------------------------ batch work queue
//
// Many independent problems whose column teams are single CTAs: one persistent launch per sweep
// direction takes (problem, column) items from a queue ordered longest first.  A CTA runs the whole
// sweep of its item, then counts the item done for its problem; the CTA that completes a problem's
// last column also reduces that problem's partials (the finalize after the forward sweep, the
// gradient reduction after the backward sweep), so no CTA ever waits for another one.
template <typename T, bool BACKWARD>
__global__ void __launch_bounds__(512, 1) k_queue(const __grid_constant__ QueueParams q) {
  __shared__ SweepParams sp;
  __shared__ int s_item, s_last;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(q.head, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= q.n_items) break;   // uniform over the CTA
    const int2 w = q.items[it];
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(q.sweep + w.x);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sp);
      for (int i = threadIdx.x; i < (int)(sizeof(SweepParams) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if constexpr (BACKWARD) backward_body<T, false>(sp, w.y);
    else forward_body<T, false>(sp, w.y);
    __threadfence();   // this CTA's partials before the count that publishes them
    __syncthreads();
    if (threadIdx.x == 0) {
      s_last = atomicAdd(q.done + w.x, 1) == sp.n_states - 1;
      __threadfence();
    }
    __syncthreads();
    if (s_last) {
      if constexpr (BACKWARD) grad_reduce_body(q.red[w.x], threadIdx.x, blockDim.x);
      else finalize_body(q.fin[w.x]);
    }
    __syncthreads();   // s_item, s_last and sp are rewritten by the next item
  }
}

// One steepest-descent update a <- a - eta grad C (Sec. II), recording the cost of the evaluation
// that produced `grad` in costs[*counter] and advancing the counter.  The update is evaluated as
// u - (eta * g) with separate roundings (no contraction), so a host can reproduce it exactly.
__global__ void k_sd_update(double* u, const double* __restrict__ grad, int64_t count, double eta,
                            const double* __restrict__ cost, double* costs, int* counter, int max_count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    u[i] = __dsub_rn(u[i], __dmul_rn(eta, grad[i]));
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int c = *counter;
    if (c < max_count) costs[c] = *cost;
    *counter = c + 1;
  }
}

cudaError_t launch_sd_update(double* u, const double* grad, int64_t count, double eta, const double* cost, double* costs,
                             int* counter, int max_count, cudaStream_t st) {
  int grid = (int)((count + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > 1024) grid = 1024;
  k_sd_update<<<grid, 256, 0, st>>>(u, grad, count, eta, cost, costs, counter, max_count);
  return cudaGetLastError();
}

__global__ void k_check_finite(const double* u, int64_t count, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(u[i])) set_error(err, kErrNonFinite);
}

// ------------------------------------------------------------------ launchers

int max_dynamic_smem(int device) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
  return v;
}

cudaError_t launch_schedule(const ScheduleParams& p, cudaStream_t st) {
  // blocks: one per step up to 1216; with fewer steps than that, rows are split into chunks of at
  // least 64 so that about 2432 blocks share the work
  int chunks = p.N >= 1216 ? 1 : std::min(std::max(1, p.dim / 64), std::max(1, 2432 / std::max(p.N, 1)));
  if (chunks <= 1) {
    const int grid = p.N < 1216 ? p.N : 1216;
    k_schedule<<<grid, 256, 0, st>>>(p);
    return cudaGetLastError();
  }
  const int rows_per = (p.dim + chunks - 1) / chunks;
  chunks = (p.dim + rows_per - 1) / rows_per;
  cudaError_t e = cudaMemsetAsync(p.norm1, 0, (size_t)p.N * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_schedule_rows<<<dim3(p.N, chunks), 256, 0, st>>>(p, rows_per);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_schedule_pick<<<(p.N + 127) / 128, 128, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename KernelT>
static cudaError_t launch_sweep(KernelT kern, const SweepParams& p, int smem_bytes, int threads, cudaStream_t st) {
  cudaError_t e = ensure_constants();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_states * p.CL);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (p.CL > 1) {
    if (p.CL > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  e = cudaLaunchKernelEx(&cfg, kern, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_forward(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st) {
  if (precision == 1) {
    if (p.CL > 1) return launch_sweep(k_forward<dw, true>, p, smem_bytes, threads, st);
    return launch_sweep(k_forward<dw, false>, p, smem_bytes, threads, st);
  }
  if (p.CL > 1) return launch_sweep(k_forward<double, true>, p, smem_bytes, threads, st);
  return launch_sweep(k_forward<double, false>, p, smem_bytes, threads, st);
}

cudaError_t launch_backward(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st) {
  if (precision == 1) {
    if (p.CL > 1) return launch_sweep(k_backward<dw, true>, p, smem_bytes, threads, st);
    return launch_sweep(k_backward<dw, false>, p, smem_bytes, threads, st);
  }
  if (p.CL > 1) return launch_sweep(k_backward<double, true>, p, smem_bytes, threads, st);
  return launch_sweep(k_backward<double, false>, p, smem_bytes, threads, st);
}

cudaError_t launch_plan(const PlanParams& p, cudaStream_t st) {
  k_plan<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename KernelT>
static cudaError_t launch_role(KernelT kern, const SweepParams& p, int blocks, int smem_bytes, int threads, int priority,
                               bool use_priority, cudaStream_t st) {
  cudaError_t e = ensure_constants();
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (p.CL > 1) {
    if (p.CL > 8) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = p.CL;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
  }
  if (use_priority) {
    attr[na].id = cudaLaunchAttributePriority;
    attr[na].val.priority = priority;
    ++na;
  }
  cfg.attrs = na ? attr : nullptr;
  cfg.numAttrs = na;
  e = cudaLaunchKernelEx(&cfg, kern, p);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_costate(const SweepParams& p, int precision, int smem_bytes, int threads, int priority,
                           cudaStream_t st) {
  const int blocks = p.n_states * p.CL;
  if (precision == 1) {
    if (p.CL > 1) return launch_role(k_costate<dw, true>, p, blocks, smem_bytes, threads, priority, true, st);
    return launch_role(k_costate<dw, false>, p, blocks, smem_bytes, threads, priority, true, st);
  }
  if (p.CL > 1) return launch_role(k_costate<double, true>, p, blocks, smem_bytes, threads, priority, true, st);
  return launch_role(k_costate<double, false>, p, blocks, smem_bytes, threads, priority, true, st);
}

cudaError_t launch_gradient(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st) {
  const int blocks = (p.n_end - p.n_begin) * p.n_states * p.CL;
  if (blocks <= 0) return cudaSuccess;
  if (precision == 1) {
    if (p.CL > 1) return launch_role(k_gradient<dw, true>, p, blocks, smem_bytes, threads, 0, false, st);
    return launch_role(k_gradient<dw, false>, p, blocks, smem_bytes, threads, 0, false, st);
  }
  if (p.CL > 1) return launch_role(k_gradient<double, true>, p, blocks, smem_bytes, threads, 0, false, st);
  return launch_role(k_gradient<double, false>, p, blocks, smem_bytes, threads, 0, false, st);
}

cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st) {
  k_finalize<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const GradReduceParams& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.K * p.N;
  int grid = (int)((total + 255) / 256);
  if (grid < 1) grid = 1;
  if (grid > 4096) grid = 4096;
  k_grad_reduce<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_schedule_batch(const ScheduleParams* ps, int count, int max_n, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int gx = 2432 / count;
  if (gx > max_n) gx = max_n;
  if (gx < 1) gx = 1;
  k_schedule_batch<<<dim3(gx, count), 256, 0, st>>>(ps);
  return cudaGetLastError();
}

using QueueKernel = void (*)(QueueParams);
static QueueKernel queue_kernel(int precision, bool backward) {
  if (precision == 1) return backward ? k_queue<dw, true> : k_queue<dw, false>;
  return backward ? k_queue<double, true> : k_queue<double, false>;
}

static cudaError_t queue_attrs(QueueKernel kern, int smem_bytes) {
  cudaError_t e = ensure_constants();
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
}

int queue_ctas_per_sm(int precision, bool backward, int threads, int smem_bytes) {
  QueueKernel kern = queue_kernel(precision, backward);
  if (queue_attrs(kern, smem_bytes) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem_bytes) != cudaSuccess) return 0;
  return n;
}

cudaError_t launch_queue(const QueueParams& q, int precision, bool backward, int ctas, int threads, int smem_bytes,
                         cudaStream_t st) {
  if (q.n_items <= 0) return cudaSuccess;
  QueueKernel kern = queue_kernel(precision, backward);
  cudaError_t e = queue_attrs(kern, smem_bytes);
  if (e != cudaSuccess) return e;
  kern<<<ctas, threads, smem_bytes, st>>>(q);
  return cudaGetLastError();
}

cudaError_t check_nonfinite_u(const double* u, int64_t count, int* err, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int grid = (int)((count + 255) / 256);
  if (grid > 1024) grid = 1024;
  k_check_finite<<<grid, 256, 0, st>>>(u, count, err);
  return cudaGetLastError();
}

}  // namespace grape
