// Eigendecomposition variant of the HG evaluation (App. F), FP64 throughout.
//
// Each step propagator is formed from a Hermitian eigendecomposition,
//     H_n = V_n diag(lambda) V_n^+,   U_n = exp(-i H_n dt) = V_n diag(exp(-i lambda dt)) V_n^+
// (App. F, Eqs. (matrix dia)), and its derivative from the divided differences of exp on the
// spectrum (App. F, Eq. (propagator der)):
//     dU_n/du_kn = V_n ( Phi o (V_n^+ (-i dt H_k) V_n) ) V_n^+,
//     Phi_ij = (e^{D_i} - e^{D_j}) / (D_i - D_j),  Phi_ii = e^{D_i},  D_i = -i lambda_i dt,
// evaluated without cancellation as exp((D_i + D_j)/2) sin(theta)/theta, theta = (lambda_i - lambda_j) dt/2.
//
// Kernels:
//   k_eig_tridiag   one CTA per step: H_n and its Householder reduction to tridiagonal form
//   k_eig_qr        one thread per step: symmetric QR steps (Wilkinson shift) on the real tridiagonal, rotations recorded
//   k_eig_rotate    one thread per row of a step: the recorded rotations applied to the identity
//   k_eig_vectors   one CTA per step: back-transformation to the eigenvectors, U_n = V diag(e) V^+
//   k_eig_forward   one CTA per column: psi_n = U_n psi_{n-1} (Eq. (statepropagation)), overlaps
//   k_eig_backward  one CTA per column: chi_{n-1} = U_n^+ chi_n + step sources (combined costate)
//   k_eig_grad      one CTA per step: G_kn = 2 Re sum_h <chi_n^h| dU_n/du_kn |psi_{n-1}^h>
// The work of the step and gradient kernels is independent across steps and fills the GPU; the
// two sweeps are the sequential part (one d x d matrix-vector product per step and column).
#include "grape_eig.h"
#include "grape_internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace grape {
namespace {

constexpr int kT = 256;
constexpr int kWarps = kT / 32;
constexpr int kQrLanes = 8;   // steps per warp in k_eig_qr (the rest of the warp idles)

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void c_fma(double2& acc, double2 a, double2 b) {   // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void c_fma_conj(double2& acc, double2 a, double2 b) {   // acc += conj(a) b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 c_conj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double warp_all_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double2 warp_all_sum2(double2 v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Sum over the block, result in every thread; warps are added in a fixed order.
__device__ double2 block_all_sum2(double2 v, double* red) {
  v = warp_all_sum2(v);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[2 * w] = v.x;
    red[2 * w + 1] = v.y;
  }
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  for (int i = 0; i < kWarps; ++i) {
    t.x += red[2 * i];
    t.y += red[2 * i + 1];
  }
  __syncthreads();
  return t;
}

// Shared-memory layout of the reduction and back-transformation kernels: one complex d x d block
// with leading dimension d + 1, three complex d-vectors and kT complex partial sums.
__host__ __device__ inline size_t block_bytes(int d) {
  return (size_t)16 * d * (d + 1) + (size_t)16 * 3 * d + (size_t)16 * kT + 8 * 2 * kWarps;
}

// Householder reduction of H_n = H0 + sum_k u_kn H_k (Sec. II) to tridiagonal form, one CTA per step.
// H_k = I - tau v v^+ maps column k below the diagonal onto alpha e_1; the trailing block B becomes
// H_k B H_k = B - v w^+ - w v^+ with p = tau B v, w = p - (tau/2)(v^+ p) v.  Writes the diagonal,
// the super-diagonal t_i = T_{i,i+1}, the vectors v_k (into the step's slice of U) and tau_k.
__global__ void __launch_bounds__(kT) k_eig_tridiag(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, step = p.step0 + blockIdx.x, tid = threadIdx.x, lda = d + 1;
  double2* A = reinterpret_cast<double2*>(sm);
  double2* vv = A + (size_t)d * lda;
  double2* pv = vv + d;
  double2* wv = pv + d;
  double2* tmp = wv + d;   // kT partial sums
  double* red = reinterpret_cast<double*>(tmp + kT);
  const size_t dd = (size_t)d * d;
  double2* hv = p.U + (size_t)step * dd;
  double* htau = p.htau + (size_t)step * d;
  for (int idx = tid; idx < d * d; idx += kT) {
    double2 h = p.H0[idx];
    for (int k = 0; k < p.K; ++k) {
      const double uk = p.u[(size_t)k * p.N + step];
      const double2 hk = p.Hk[(size_t)k * dd + idx];
      h.x = fma(uk, hk.x, h.x);
      h.y = fma(uk, hk.y, h.y);
    }
    A[(idx / d) * lda + idx % d] = h;
  }
  __syncthreads();
  for (int k = 0; k + 2 < d; ++k) {
    const int n1 = d - k - 1;
    double2 part = make_double2(0.0, 0.0);
    for (int i = 1 + tid; i < n1; i += kT) {
      const double2 x = A[(k + 1 + i) * lda + k];
      part.x = fma(x.x, x.x, fma(x.y, x.y, part.x));
    }
    const double sigma = block_all_sum2(part, red).x;
    const double2 x0 = A[(k + 1) * lda + k];
    double tau = 0.0;
    double2 alpha = x0, v0 = make_double2(0.0, 0.0);
    if (sigma > 0.0) {
      const double ax0 = hypot(x0.x, x0.y);
      const double xn = sqrt(fma(ax0, ax0, sigma));
      const double2 phs = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      alpha = make_double2(-phs.x * xn, -phs.y * xn);
      tau = 1.0 / (xn * (xn + ax0));
      v0 = make_double2(phs.x * (ax0 + xn), phs.y * (ax0 + xn));
    }
    if (tau != 0.0) {
      for (int i = tid; i < n1; i += kT) {
        const double2 vi = i == 0 ? v0 : A[(k + 1 + i) * lda + k];
        vv[i] = vi;
        hv[(size_t)k * d + i] = vi;
      }
      __syncthreads();
      {   // p_i = tau sum_j B_ij v_j = tau sum_j conj(B_ji) v_j: rows of B read along i, j split in chunks
        const int parts = kT / n1 < 1 ? 1 : kT / n1;
        for (int t = tid; t < parts * n1; t += kT) {
          const int i = t % n1, q = t / n1;
          const int j0 = (int)((int64_t)q * n1 / parts), j1 = (int)((int64_t)(q + 1) * n1 / parts);
          double2 acc = make_double2(0.0, 0.0);
          for (int j = j0; j < j1; ++j) c_fma_conj(acc, A[(k + 1 + j) * lda + (k + 1 + i)], vv[j]);
          tmp[t] = acc;
        }
        __syncthreads();
        for (int i = tid; i < n1; i += kT) {
          double2 acc = tmp[i];
          for (int q = 1; q < parts; ++q) {
            acc.x += tmp[q * n1 + i].x;
            acc.y += tmp[q * n1 + i].y;
          }
          pv[i] = make_double2(tau * acc.x, tau * acc.y);
        }
      }
      __syncthreads();
      double2 vp = make_double2(0.0, 0.0);
      for (int i = tid; i < n1; i += kT) vp.x = fma(vv[i].x, pv[i].x, fma(vv[i].y, pv[i].y, vp.x));
      const double kc = 0.5 * tau * block_all_sum2(vp, red).x;
      for (int i = tid; i < n1; i += kT) wv[i] = make_double2(fma(-kc, vv[i].x, pv[i].x), fma(-kc, vv[i].y, pv[i].y));
      __syncthreads();
      for (int idx = tid; idx < n1 * n1; idx += kT) {
        const int i = idx / n1, j = idx % n1;
        double2& b = A[(k + 1 + i) * lda + (k + 1 + j)];
        const double2 vi = vv[i], wi = wv[i], vj = vv[j], wj = wv[j];
        // b -= v_i conj(w_j) + w_i conj(v_j)
        b.x -= vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
        b.y -= vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
      }
    }
    if (tid == 0) {
      htau[k] = tau;
      A[(k + 1) * lda + k] = alpha;
      A[k * lda + (k + 1)] = c_conj(alpha);
    }
    __syncthreads();
  }
  for (int i = tid; i < d; i += kT) {
    p.tri_a[(size_t)step * d + i] = A[i * lda + i].x;
    p.tri_t[(size_t)step * d + i] = i + 1 < d ? A[i * lda + i + 1] : make_double2(0.0, 0.0);
  }
}

// Eigenvalues of the real symmetric tridiagonal T_r = P^+ T P (P diagonal phases,
// P_{i+1} = P_i conj(t_i)/|t_i|) by the symmetric QR algorithm with implicit Wilkinson-shifted steps
// (Golub & Van Loan, Matrix Computations, 4th ed., Sec. 8.3: Algorithm 8.3.2 for one step,
// Algorithm 8.3.3 for deflation).  The unreduced block [lo, hi] at the bottom of the part not yet
// converged gets one step at a time:
//   * shift mu = the eigenvalue of its trailing 2x2 block closer to a_hi;
//   * the first rotation maps the first column of T - mu I, (a_lo - mu, b_lo), onto its norm;
//   * each rotation R_k = [[c, s], [-s, c]] on rows/columns k, k+1 (T <- R_k T R_k^T) turns the
//     entry b_{k+1} below it into a bulge at (k, k+2), which the next rotation removes; the last
//     rotation leaves T tridiagonal again;
//   * an off-diagonal |b_i| <= u (|a_i| + |a_{i+1}|) is set to zero, which splits the matrix; a zero
//     at the bottom of the block (hi) frees the eigenvalue a_hi.
// One thread per step: GB300 retires a warp's FP64 instruction only every few tens of clocks per
// SM sub-partition, so the sequential scalar recurrence runs with kQrLanes steps side by side in
// the lanes of a warp, spread over many SMs.  Every rotation is recorded (index k, c, s) for
// k_eig_rotate, the eigenvalues go to lam.  At most kMaxQrSteps steps per eigenvalue and p.rot_cap
// rotations per step; past either limit kErrEig is set.
constexpr int kMaxQrSteps = 60;

__device__ __forceinline__ bool offdiag_negligible(double b, double a0, double a1) {
  return fabs(b) <= 0x1p-53 * (fabs(a0) + fabs(a1));
}

__global__ void __launch_bounds__(32) k_eig_qr(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, lane = threadIdx.x, step = p.step0 + blockIdx.x * kQrLanes + lane;
  if (lane >= kQrLanes || step >= p.step0 + p.nsteps) return;   // no block-wide synchronisation here
  // the lane's diagonal dg[i * 32] and off-diagonal od[i * 32] = T_r[i][i+1], interleaved by lane
  double* dg = reinterpret_cast<double*>(sm) + lane;
  double* od = dg + 32 * d;
  const double* ta = p.tri_a + (size_t)step * d;
  const double2* tt = p.tri_t + (size_t)step * d;
  double2* ph = p.phase + (size_t)step * d;
  double2 phi = make_double2(1.0, 0.0);
  for (int i = 0; i < d; ++i) {
    dg[i * 32] = ta[i];
    ph[i] = phi;
    double mag = 0.0;
    if (i + 1 < d) {
      const double2 t = tt[i];
      mag = hypot(t.x, t.y);
      if (mag > 0.0) phi = c_mul(phi, make_double2(t.x / mag, -t.y / mag));
    }
    od[i * 32] = mag;
  }
  const int cap = p.rot_cap;
  int* ri = p.rot_i + (size_t)step * cap;
  double2* rcs = p.rot_cs + (size_t)step * cap;
  int nrot = 0, steps_here = 0;
  bool failed = false;
  int hi = d - 1;
  while (hi > 0) {
    if (offdiag_negligible(od[(hi - 1) * 32], dg[(hi - 1) * 32], dg[hi * 32])) {
      od[(hi - 1) * 32] = 0.0;   // a_hi is an eigenvalue
      --hi;
      steps_here = 0;
      continue;
    }
    int lo = hi - 1;   // top of the unreduced block that ends at hi
    while (lo > 0 && !offdiag_negligible(od[(lo - 1) * 32], dg[(lo - 1) * 32], dg[lo * 32])) --lo;
    if (lo > 0) od[(lo - 1) * 32] = 0.0;
    if (++steps_here > kMaxQrSteps) {
      failed = true;
      break;
    }
    // Wilkinson shift: eigenvalue of [[a_{hi-1}, b], [b, a_hi]] closer to a_hi
    const double half_gap = 0.5 * (dg[(hi - 1) * 32] - dg[hi * 32]);
    const double bt = od[(hi - 1) * 32];
    const double mu = dg[hi * 32] - bt * (bt / (half_gap + copysign(hypot(half_gap, bt), half_gap)));
    double x = dg[lo * 32] - mu, z = od[lo * 32];
    for (int k = lo; k < hi; ++k) {
      const double r = hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
      if (k > lo) od[(k - 1) * 32] = r;   // the bulge at (k - 1, k + 1) is gone
      const double a0 = dg[k * 32], a1 = dg[(k + 1) * 32], b0 = od[k * 32];
      const double cc = c * c, ss = s * s, cs2 = 2.0 * c * s;
      dg[k * 32] = cc * a0 + cs2 * b0 + ss * a1;
      dg[(k + 1) * 32] = ss * a0 - cs2 * b0 + cc * a1;
      od[k * 32] = c * s * (a1 - a0) + (cc - ss) * b0;
      if (k + 1 < hi) {
        const double b1 = od[(k + 1) * 32];
        z = s * b1;                   // new bulge at (k, k + 2)
        od[(k + 1) * 32] = c * b1;
      }
      x = od[k * 32];
      if (nrot < cap) {
        ri[nrot] = k;
        rcs[nrot] = make_double2(c, s);
      }
      ++nrot;
    }
  }
  if (failed || nrot > cap) atomicCAS(p.err, 0, kErrEig);
  p.rot_n[step] = nrot < cap ? nrot : cap;
  for (int i = 0; i < d; ++i) p.lam[(size_t)step * d + i] = dg[i * 32];
}

// Eigenvectors of T_r: T_r = Q diag(lam) Q^T with Q = R_1^T R_2^T ..., the recorded rotations in
// order; every thread forms its own row of Q (the rows are independent), z <- z R_k^T on entries
// k, k+1, then Y = P Q is written to the step's slice of V.
__global__ void __launch_bounds__(128) k_eig_rotate(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, step = p.step0 + blockIdx.x, row = threadIdx.x;
  if (row >= d) return;   // no block-wide synchronisation in this kernel
  double* z = reinterpret_cast<double*>(sm) + (size_t)row * (d + 1);
  for (int c = 0; c < d; ++c) z[c] = c == row ? 1.0 : 0.0;
  const int n = p.rot_n[step];
  const int* ri = p.rot_i + (size_t)step * p.rot_cap;
  const double2* rcs = p.rot_cs + (size_t)step * p.rot_cap;
  for (int r = 0; r < n; ++r) {
    const int i = ri[r];
    const double2 cs = rcs[r];
    const double z0 = z[i], z1 = z[i + 1];
    z[i] = fma(cs.x, z0, cs.y * z1);
    z[i + 1] = fma(cs.x, z1, -cs.y * z0);
  }
  const double2 ph = p.phase[(size_t)step * d + row];
  double2* y = p.V + (size_t)step * d * d + (size_t)row * d;
  for (int c = 0; c < d; ++c) y[c] = make_double2(ph.x * z[c], ph.y * z[c]);
}

// Back-transformation V_n = H_0 H_1 ... H_{d-3} Y (right to left), the transposed copy, and
// U_n = V_n diag(exp(-i lambda dt)) V_n^+ written over the step's Householder vectors.
__global__ void __launch_bounds__(kT) k_eig_vectors(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, step = p.step0 + blockIdx.x, tid = threadIdx.x, lda = d + 1;
  double2* A = reinterpret_cast<double2*>(sm);
  double2* vv = A + (size_t)d * lda;
  double2* pv = vv + d;
  double2* tmp = pv + 2 * d;   // kT partial sums (same layout as the reduction kernel)
  const size_t dd = (size_t)d * d;
  const double2* hv = p.U + (size_t)step * dd;
  const double* htau = p.htau + (size_t)step * d;
  double2* V = p.V + (size_t)step * dd;
  for (int idx = tid; idx < d * d; idx += kT) A[(idx / d) * lda + idx % d] = V[idx];
  __syncthreads();
  // H_k Y = Y - tau v (v^+ Y) on rows k+1..d-1: thread (c, q) sums rows of chunk q of column c,
  // then subtracts from the same rows; the chunk sums of a column meet in tmp.
  const int parts = kT / d < 1 ? 1 : kT / d;
  for (int k = d - 3; k >= 0; --k) {
    const double tau = htau[k];
    if (tau == 0.0) continue;
    const int n1 = d - k - 1;
    for (int i = tid; i < n1; i += kT) vv[i] = hv[(size_t)k * d + i];
    __syncthreads();
    const int c = tid % d, q = tid / d;
    const bool active = q < parts;
    const int i0 = (int)((int64_t)q * n1 / parts), i1 = (int)((int64_t)(q + 1) * n1 / parts);
    if (active) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = i0; i < i1; ++i) c_fma_conj(acc, vv[i], A[(k + 1 + i) * lda + c]);
      tmp[tid] = acc;
    }
    __syncthreads();
    if (active) {
      double2 sc = tmp[c];
      for (int r = 1; r < parts; ++r) {
        sc.x += tmp[r * d + c].x;
        sc.y += tmp[r * d + c].y;
      }
      sc.x *= tau;
      sc.y *= tau;
      for (int i = i0; i < i1; ++i) {
        double2& y = A[(k + 1 + i) * lda + c];
        const double2 t = c_mul(vv[i], sc);
        y.x -= t.x;
        y.y -= t.y;
      }
    }
    __syncthreads();
  }
  const double* lam = p.lam + (size_t)step * d;
  double2* Vt = p.Vt + (size_t)step * dd;
  for (int i = tid; i < d; i += kT) {
    double sn, cs;
    sincos(lam[i] * p.dt, &sn, &cs);
    pv[i] = make_double2(cs, -sn);
  }
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, c = idx % d;
    const double2 y = A[i * lda + c];
    V[idx] = y;
    Vt[(size_t)c * d + i] = y;
  }
  __syncthreads();   // every read of the Householder vectors is done
  double2* U = p.U + (size_t)step * dd;
  constexpr int kJ = 4;   // entries U_ij, j = j0 .. j0 + 3, per thread share the product Y_il e_l
  const int nj = (d + kJ - 1) / kJ;
  for (int w = tid; w < d * nj; w += kT) {
    const int i = w / nj, j0 = (w % nj) * kJ;
    const double2* yi = A + i * lda;
    double2 acc[kJ];
#pragma unroll
    for (int q = 0; q < kJ; ++q) acc[q] = make_double2(0.0, 0.0);
    for (int l = 0; l < d; ++l) {
      const double2 a = c_mul(yi[l], pv[l]);
#pragma unroll
      for (int q = 0; q < kJ; ++q)
        if (j0 + q < d) c_fma(acc[q], a, c_conj(A[(j0 + q) * lda + l]));
    }
#pragma unroll
    for (int q = 0; q < kJ; ++q)
      if (j0 + q < d) U[(size_t)i * d + j0 + q] = acc[q];
  }
}

// Rows [row_begin(q), row_begin(q + 1)) of a column belong to CTA q of the column's cluster.
__device__ __forceinline__ int row_begin(int q, int d, int cl) { return (int)((int64_t)q * d / cl); }

__device__ __forceinline__ int row_owner(int i, int d, int cl) {
  int q = (int)((int64_t)i * cl / d);
  while (q + 1 < cl && row_begin(q + 1, d, cl) <= i) ++q;
  while (q > 0 && row_begin(q, d, cl) > i) --q;
  return q;
}

// The rows computed by the other CTAs of the cluster, read from their copy of `buf` (same offset).
template <bool CLUSTER>
__device__ __forceinline__ void exchange_rows(double2* buf, int d, int cl, int rank, int r0, int r1) {
  if constexpr (CLUSTER) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();   // every CTA's own rows of buf are written
    for (int i = threadIdx.x; i < d; i += kT) {
      if (i >= r0 && i < r1) continue;
      buf[i] = *cluster.map_shared_rank(buf + i, row_owner(i, d, cl));
    }
  }
  __syncthreads();
}

// Forward sweep of column h = blockIdx.x / CL over steps [p.step0, p.step0 + p.nsteps), rows split
// over a cluster of CL CTAs: psi_s = U_s psi_{s-1} (Eq. (statepropagation)); overlaps and the C2 /
// C3 accumulations per CTA (C2 partials add up over the launches of one sweep).  Double-buffered: a
// CTA rewrites a buffer two steps after it was read remotely, and the cluster barrier of the step in
// between orders the two.
template <bool CLUSTER>
__global__ void __launch_bounds__(kT) k_eig_forward(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, cl = p.sweep_cl, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int h = blockIdx.x / cl, rank = blockIdx.x % cl, part = h * cl + rank;
  const int r0 = row_begin(rank, d, cl), r1 = row_begin(rank + 1, d, cl);
  double2* buf0 = reinterpret_cast<double2*>(sm);
  double2* buf1 = buf0 + d;
  double* red = reinterpret_cast<double*>(buf1 + d);
  const size_t dd = (size_t)d * d, col = (size_t)h * d, slab = (size_t)p.n * d;
  const double2* tgt = p.target + col;
  const int s0 = p.step0, s1 = p.step0 + p.nsteps;
  const double2* start = s0 == 0 ? p.psi0 + col : p.psi_hist + (size_t)s0 * slab + col;
  for (int i = tid; i < d; i += kT) buf0[i] = start[i];
  if (s0 == 0)
    for (int i = r0 + tid; i < r1; i += kT) p.psi_hist[col + i] = p.psi0[col + i];
  __syncthreads();
  double c2 = 0.0;
  for (int s = s0; s < s1; ++s) {
    const double2* cur = ((s - s0) & 1) ? buf1 : buf0;
    double2* nxt = ((s - s0) & 1) ? buf0 : buf1;
    const double2* Us = p.U + (size_t)s * dd;
    double2* hist = p.psi_hist + (size_t)(s + 1) * slab + col;
    for (int i = r0 + warp; i < r1; i += kWarps) {
      const double2* urow = Us + (size_t)i * d;
      double2 acc = make_double2(0.0, 0.0);
      for (int j = lane; j < d; j += 32) c_fma(acc, urow[j], cur[j]);
      acc = warp_all_sum2(acc);
      if (lane == 0) {
        nxt[i] = acc;
        hist[i] = acc;
        if (p.omega) c2 = fma(p.omega[i], fma(acc.x, acc.x, acc.y * acc.y), c2);
      }
    }
    exchange_rows<CLUSTER>(nxt, d, cl, rank, r0, r1);
    if (p.part_g3) {
      double2 g = make_double2(0.0, 0.0);
      for (int i = r0 + tid; i < r1; i += kT) c_fma_conj(g, tgt[i], nxt[i]);
      g = block_all_sum2(g, red);
      if (tid == 0) p.part_g3[(size_t)part * p.N + s] = g;
    }
  }
  const double2* fin = ((s1 - s0) & 1) ? buf1 : buf0;
  double2 g = make_double2(0.0, 0.0);
  for (int i = r0 + tid; i < r1; i += kT) c_fma_conj(g, tgt[i], fin[i]);
  g = block_all_sum2(g, red);
  const double c2s = block_all_sum2(make_double2(c2, 0.0), red).x;
  if (tid == 0) {
    p.part_g[part] = g;   // the overlap of the sweep's last state (the last launch writes it last)
    p.part_c2[part] = s0 == 0 ? c2s : p.part_c2[part] + c2s;
  }
  if constexpr (CLUSTER) cg::this_cluster().sync();   // no CTA leaves while its rows may still be read
}

// Backward sweep of column h (rows split over the cluster as in the forward sweep): the combined costate
//   chi_N = -(w_fid g / n^2) phi_T + (w_forbid/(N n)) Omega psi_N - (w_tint/(N n^2)) g_N phi_T,
//   chi_{s-1} = U_s^+ chi_s + (w_forbid/(N n)) Omega psi_{s-1} - (w_tint/(N n^2)) g_{s-1} phi_T.
template <bool CLUSTER>
__global__ void __launch_bounds__(kT) k_eig_backward(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, cl = p.sweep_cl, tid = threadIdx.x;
  const int h = blockIdx.x / cl, rank = blockIdx.x % cl;
  const int r0 = row_begin(rank, d, cl), r1 = row_begin(rank + 1, d, cl), nr = r1 - r0;
  const int parts = nr > 0 ? (kT / nr < 1 ? 1 : (kT / nr > d ? d : kT / nr)) : 1;
  double2* buf0 = reinterpret_cast<double2*>(sm);
  double2* buf1 = buf0 + d;
  double2* tmp = buf1 + d;   // parts x nr partial products
  const size_t dd = (size_t)d * d, col = (size_t)h * d, slab = (size_t)p.n * d;
  const double2* tgt = p.target + col;
  const double nS = (double)p.n, Nd = (double)p.N;
  const double2 g = *p.g_final;
  double2 coef = make_double2(-p.w_fid * g.x / (nS * nS), -p.w_fid * g.y / (nS * nS));
  const double c3w = p.w_tint != 0.0 ? -p.w_tint / (Nd * nS * nS) : 0.0;
  if (c3w != 0.0) {
    coef.x = fma(c3w, p.g3[p.N - 1].x, coef.x);
    coef.y = fma(c3w, p.g3[p.N - 1].y, coef.y);
  }
  const double c2w = (p.omega && p.w_forbid != 0.0) ? p.w_forbid / (Nd * nS) : 0.0;
  {
    const double2* psiN = p.psi_hist + (size_t)p.N * slab + col;
    double2* hist = p.chi_hist + (size_t)p.N * slab + col;
    for (int i = tid; i < d; i += kT) {
      double2 ch = c_mul(coef, tgt[i]);
      if (c2w != 0.0) {
        const double w = c2w * p.omega[i];
        ch.x = fma(w, psiN[i].x, ch.x);
        ch.y = fma(w, psiN[i].y, ch.y);
      }
      buf0[i] = ch;
      if (i >= r0 && i < r1) hist[i] = ch;
    }
  }
  __syncthreads();
  for (int s = p.N; s >= 2; --s) {
    const int it = p.N - s;
    const double2* cur = (it & 1) ? buf1 : buf0;
    double2* nxt = (it & 1) ? buf0 : buf1;
    const double2* Us = p.U + (size_t)(s - 1) * dd;
    for (int t = tid; t < parts * nr; t += kT) {
      const int i = r0 + t % nr, q = t / nr;
      const int j0 = (int)((int64_t)q * d / parts), j1 = (int)((int64_t)(q + 1) * d / parts);
      double2 acc = make_double2(0.0, 0.0);
      for (int j = j0; j < j1; ++j) c_fma_conj(acc, Us[(size_t)j * d + i], cur[j]);
      tmp[t] = acc;
    }
    __syncthreads();
    const double2* psi = p.psi_hist + (size_t)(s - 1) * slab + col;
    double2* hist = p.chi_hist + (size_t)(s - 1) * slab + col;
    double2 c3 = make_double2(0.0, 0.0);
    if (c3w != 0.0) c3 = make_double2(c3w * p.g3[s - 2].x, c3w * p.g3[s - 2].y);
    for (int li = tid; li < nr; li += kT) {
      const int i = r0 + li;
      double2 y = tmp[li];
      for (int q = 1; q < parts; ++q) {
        y.x += tmp[(size_t)q * nr + li].x;
        y.y += tmp[(size_t)q * nr + li].y;
      }
      if (c2w != 0.0) {
        const double w = c2w * p.omega[i];
        y.x = fma(w, psi[i].x, y.x);
        y.y = fma(w, psi[i].y, y.y);
      }
      if (c3w != 0.0) c_fma(y, c3, tgt[i]);
      nxt[i] = y;
      hist[i] = y;
    }
    exchange_rows<CLUSTER>(nxt, d, cl, rank, r0, r1);
  }
  if constexpr (CLUSTER) cg::this_cluster().sync();
}

// sin(x)/x: the Taylor series of sin(x)/x through x^12 for |x| < 1/4 (remainder below 1e-20),
// else the ratio itself.
__device__ __forceinline__ double sinc_of(double x, double sin_x) {
  if (fabs(x) < 0.25) {
    const double x2 = x * x;
    double t = 1.0 / 6227020800.0;           // 1/13!
    t = fma(t, x2, -1.0 / 39916800.0);       // 1/11!
    t = fma(t, x2, 1.0 / 362880.0);          // 1/9!
    t = fma(t, x2, -1.0 / 5040.0);           // 1/7!
    t = fma(t, x2, 1.0 / 120.0);             // 1/5!
    t = fma(t, x2, -1.0 / 6.0);              // 1/3!
    return fma(t, x2, 1.0);
  }
  return sin_x / x;
}

// Phi_ij = exp((D_i + D_j)/2) sin(theta)/theta with D = -i lambda dt and theta = alpha_i - alpha_j,
// alpha = lambda dt / 2, from the per-eigenvalue cos/sin of alpha: exp((D_i + D_j)/2) = h_i h_j with
// h = (cos alpha, -sin alpha), sin(theta) = s_i c_j - c_i s_j (used only where |theta| >= 1/4).
__device__ __forceinline__ double2 divided_difference(double ai, double aj, double ci, double si, double cj,
                                                      double sj) {
  const double th = ai - aj;
  const double sinc = sinc_of(th, fma(si, cj, -ci * sj));
  const double2 hh = c_mul(make_double2(ci, -si), make_double2(cj, -sj));
  return make_double2(hh.x * sinc, hh.y * sinc);
}

// Gradient of step s + 1 (block s):  with psi' = V^+ psi_s and chi' = V^+ chi_{s+1} (V = V_{s+1}),
//   Q = Phi o M,  M_ij = sum_h conj(chi'_hi) psi'_hj,
//   sum_h <chi^h| dU/du_k |psi^h> = -i dt sum_ab H_k,ab T_ab,  T = conj(V) Q V^T,
// so G_k = 2 dt Im(sum_ab H_k,ab T_ab).  T is formed one column b at a time per warp
// (c = Q V_b^T, then T_:b = conj(V) c) and contracted with every H_k at once.
__global__ void __launch_bounds__(kT, 1) k_eig_grad(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n = p.n, K = p.K;
  const int ldq = d + 1;
  double2* Q = reinterpret_cast<double2*>(sm);
  double2* cw = Q + (size_t)d * ldq;                       // kWarps x d
  double* acck = reinterpret_cast<double*>(cw + (size_t)kWarps * d);   // kWarps x K
  double* ha = acck + kWarps * (K > 0 ? K : 1);                        // alpha_i = lambda_i dt / 2
  double* hc = ha + d;                                                 // cos alpha_i
  double* hs = hc + d;                                                 // sin alpha_i
  const size_t dd = (size_t)d * d, slab = (size_t)n * d;
  const double2* V = p.V + (size_t)s * dd;
  const double2* Vt = p.Vt + (size_t)s * dd;
  const double* lam = p.lam + (size_t)s * d;
  const double2* psi = p.psi_hist + (size_t)s * slab;
  const double2* chi = p.chi_hist + (size_t)(s + 1) * slab;
  double2* xp = p.xs + (size_t)s * 2 * slab;
  double2* xc = xp + slab;
  for (int idx = tid; idx < n * d; idx += kT) {
    const int h = idx / d, i = idx % d;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    for (int j = 0; j < d; ++j) {
      const double2 vji = V[(size_t)j * d + i];
      c_fma_conj(a, vji, psi[(size_t)h * d + j]);
      c_fma_conj(b, vji, chi[(size_t)h * d + j]);
    }
    xp[idx] = a;
    xc[idx] = b;
  }
  for (int i = tid; i < kWarps * K; i += kT) acck[i] = 0.0;
  for (int i = tid; i < d; i += kT) {
    const double al = 0.5 * lam[i] * p.dt;
    ha[i] = al;
    sincos(al, &hs[i], &hc[i]);
  }
  __syncthreads();
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, j = idx % d;
    double2 m = make_double2(0.0, 0.0);
    for (int h = 0; h < n; ++h) c_fma_conj(m, xc[(size_t)h * d + i], xp[(size_t)h * d + j]);
    Q[i * ldq + j] = c_mul(divided_difference(ha[i], ha[j], hc[i], hs[i], hc[j], hs[j]), m);
  }
  __syncthreads();
  double2* c = cw + (size_t)warp * d;
  for (int b = warp; b < d; b += kWarps) {
    const double2* vb = V + (size_t)b * d;
    for (int i = lane; i < d; i += 32) {
      const double2* qi = Q + i * ldq;
      double2 acc = make_double2(0.0, 0.0);
      for (int j = 0; j < d; ++j) c_fma(acc, qi[j], vb[j]);
      c[i] = acc;
    }
    __syncwarp();
    // T_ab only where some H_k[a][b] != 0 (column b of the controls' union pattern, at most d rows)
    constexpr int kPer = (kEigMaxDim + 31) / 32;   // pattern entries e0 + lane + 32 q held per lane
    const int e0 = p.cp_ptr[b], ne = p.cp_ptr[b + 1] - e0;
    double2 t[kPer];
    int arow[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = lane + 32 * q;
      double2 acc = make_double2(0.0, 0.0);
      arow[q] = 0;
      if (e < ne) {
        const int a = p.cp_row[e0 + e];
        arow[q] = a;
        for (int i = 0; i < d; ++i) c_fma_conj(acc, Vt[(size_t)i * d + a], c[i]);
      }
      t[q] = acc;
    }
    for (int k = 0; k < K; ++k) {
      const double2* hb = p.Hk + (size_t)k * dd + (size_t)b * d;   // H_k[b][a] = conj(H_k[a][b])
      double im = 0.0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        if (lane + 32 * q < ne) {
          const double2 hba = hb[arow[q]];
          im = fma(hba.x, t[q].y, fma(-hba.y, t[q].x, im));
        }
      }
      im = warp_all_sum(im);
      if (lane == 0) acck[warp * K + k] += im;
    }
    __syncwarp();
  }
  __syncthreads();
  for (int k = tid; k < K; k += kT) {
    double im = 0.0;
    for (int w = 0; w < kWarps; ++w) im += acck[w * K + k];
    p.part_grad[(size_t)s * K + k] = 2.0 * p.dt * im;
  }
}

size_t forward_smem(int d) { return (size_t)16 * 2 * d + 8 * 2 * kWarps; }
size_t backward_smem(int d) { return (size_t)16 * (2 * d + kT); }

}  // namespace

int eig_step_smem(int d) { return (int)block_bytes(d); }

int eig_qr_smem(int d) { return 8 * 2 * 32 * d; }

int eig_rotate_smem(int d) { return 8 * d * (d + 1); }

int eig_grad_smem(int d, int K) {
  return (int)((size_t)16 * d * (d + 1) + (size_t)16 * kWarps * d + (size_t)8 * kWarps * (K > 0 ? K : 1) +
               (size_t)8 * 3 * d);
}

cudaError_t eig_prepare(int d, int K) {
  cudaError_t e = cudaFuncSetAttribute(k_eig_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_step_smem(d));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eig_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_step_smem(d));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_eig_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_qr_smem(d));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eig_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_rotate_smem(d));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eig_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_grad_smem(d, K));
  return e;
}

template <typename KernelT>
cudaError_t launch_sweep_kernel(KernelT kern, const EigCtx& c, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.n * c.sweep_cl);
  cfg.blockDim = dim3(kT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (c.sweep_cl > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c.sweep_cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, c);
}

cudaError_t eig_propagators(const EigCtx& c, cudaStream_t st) {
  k_eig_tridiag<<<c.nsteps, kT, eig_step_smem(c.d), st>>>(c);
  k_eig_qr<<<(c.nsteps + kQrLanes - 1) / kQrLanes, 32, eig_qr_smem(c.d), st>>>(c);
  k_eig_rotate<<<c.nsteps, (c.d + 31) / 32 * 32, eig_rotate_smem(c.d), st>>>(c);
  k_eig_vectors<<<c.nsteps, kT, eig_step_smem(c.d), st>>>(c);
  return cudaGetLastError();
}

cudaError_t eig_forward_sweep(const EigCtx& c, cudaStream_t st) {
  const size_t smem = forward_smem(c.d);
  return c.sweep_cl > 1 ? launch_sweep_kernel(k_eig_forward<true>, c, smem, st)
                        : launch_sweep_kernel(k_eig_forward<false>, c, smem, st);
}

cudaError_t eig_backward(const EigCtx& c, cudaStream_t st) {
  const size_t smem = backward_smem(c.d);
  cudaError_t e = c.sweep_cl > 1 ? launch_sweep_kernel(k_eig_backward<true>, c, smem, st)
                                 : launch_sweep_kernel(k_eig_backward<false>, c, smem, st);
  if (e != cudaSuccess || c.K == 0) return e;
  k_eig_grad<<<c.N, kT, eig_grad_smem(c.d, c.K), st>>>(c);
  return cudaGetLastError();
}

}  // namespace grape
