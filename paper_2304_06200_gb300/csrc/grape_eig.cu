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
// Kernels (all launched with 256 threads):
//   k_eig_step      one CTA per step: H_n, Householder reduction to real tridiagonal form, implicit
//                   QL on the tridiagonal (one warp), back-transformation, U_n = V diag(e) V^+
//   k_eig_forward   one CTA per column: psi_n = U_n psi_{n-1} (Eq. (statepropagation)), overlaps
//   k_eig_backward  one CTA per column: chi_{n-1} = U_n^+ chi_n + step sources (combined costate)
//   k_eig_grad      one CTA per step: G_kn = 2 Re sum_h <chi_n^h| dU_n/du_kn |psi_{n-1}^h>
// The work of the step and gradient kernels is independent across steps and fills the GPU; the
// two sweeps are the sequential part (one d x d matrix-vector product per step and column).
#include "grape_eig.h"
#include "grape_internal.h"

namespace grape {
namespace {

constexpr int kT = 256;
constexpr int kWarps = kT / 32;

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

struct StepLayout {
  int lda;            // leading dimension (d + 1) of the d x d blocks
  size_t a, z, v, p, w, ph, ad, ed, red, bytes;
};

__host__ __device__ inline StepLayout step_layout(int d) {
  StepLayout L;
  L.lda = d + 1;
  size_t off = 0;
  L.a = off;  off += (size_t)16 * d * L.lda;    // complex A, later the eigenvector block Y
  L.z = off;  off += (size_t)8 * d * L.lda;     // real Z (eigenvectors of the tridiagonal)
  off = (off + 15) & ~(size_t)15;
  L.v = off;  off += (size_t)16 * d;
  L.p = off;  off += (size_t)16 * d;
  L.w = off;  off += (size_t)16 * d;
  L.ph = off; off += (size_t)16 * d;
  L.ad = off; off += (size_t)8 * d;
  L.ed = off; off += (size_t)8 * d;
  L.red = off; off += (size_t)8 * 2 * kWarps;
  L.bytes = off;
  return L;
}

// Implicit QL with Wilkinson-type shifts on the real symmetric tridiagonal (a, e), e[i] coupling
// rows i and i+1, accumulating the plane rotations into the columns of Z (textbook algorithm for
// symmetric tridiagonal eigenproblems).  Run by one warp: every lane evaluates the same scalar
// recurrence, lane 0 alone stores a and e (followed by __syncwarp), and each lane rotates its own
// rows of Z.  Gives up after 60 iterations for one eigenvalue and sets kErrEig.
__device__ void tridiagonal_ql(double* a, double* e, double* Z, int d, int lda, int* err) {
  const int lane = threadIdx.x & 31;
  for (int l = 0; l < d; ++l) {
    int iter = 0;
    for (;;) {
      int m = l;
      for (; m < d - 1; ++m) {
        const double dd = fabs(a[m]) + fabs(a[m + 1]);
        if (fabs(e[m]) + dd == dd) break;
      }
      if (m == l) break;
      if (++iter > 60) {
        if (lane == 0) atomicCAS(err, 0, kErrEig);
        break;
      }
      double g = (a[l + 1] - a[l]) / (2.0 * e[l]);
      double r = hypot(g, 1.0);
      g = a[m] - a[l] + e[l] / (g + copysign(r, g));
      double s = 1.0, c = 1.0, shift = 0.0;
      bool split = false;
      for (int i = m - 1; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = hypot(f, g);
        if (lane == 0) e[i + 1] = r;
        if (r == 0.0) {   // underflow: the off-diagonal element splits the matrix here
          const double ai1 = a[i + 1] - shift;
          __syncwarp();
          if (lane == 0) {
            a[i + 1] = ai1;
            e[m] = 0.0;
          }
          __syncwarp();
          split = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = a[i + 1] - shift;
        r = (a[i] - g) * s + 2.0 * c * b;
        shift = s * r;
        const double ai1 = g + shift;
        g = c * r - b;
        for (int row = lane; row < d; row += 32) {
          double* zr = Z + (size_t)row * lda;
          const double z1 = zr[i + 1], z0 = zr[i];
          zr[i + 1] = s * z0 + c * z1;
          zr[i] = c * z0 - s * z1;
        }
        __syncwarp();
        if (lane == 0) a[i + 1] = ai1;
        __syncwarp();
      }
      if (split) continue;
      const double al = a[l] - shift;
      __syncwarp();
      if (lane == 0) {
        a[l] = al;
        e[l] = g;
        e[m] = 0.0;
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(kT, 1) k_eig_step(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, step = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const StepLayout L = step_layout(d);
  const int lda = L.lda;
  double2* A = reinterpret_cast<double2*>(sm + L.a);
  double* Z = reinterpret_cast<double*>(sm + L.z);
  double2* vv = reinterpret_cast<double2*>(sm + L.v);
  double2* pv = reinterpret_cast<double2*>(sm + L.p);
  double2* wv = reinterpret_cast<double2*>(sm + L.w);
  double2* ph = reinterpret_cast<double2*>(sm + L.ph);
  double* ad = reinterpret_cast<double*>(sm + L.ad);
  double* ed = reinterpret_cast<double*>(sm + L.ed);
  double* red = reinterpret_cast<double*>(sm + L.red);
  const size_t dd = (size_t)d * d;
  double2* hv = p.U + (size_t)step * dd;      // Householder vectors of this step (row k: v_k)
  double* htau = p.htau + (size_t)step * d;

  // H_n = H0 + sum_k u_kn H_k (Sec. II)
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

  // Householder reduction: H_k = I - tau v v^+ maps column k below the diagonal onto alpha e_1;
  // the trailing block B becomes H_k B H_k = B - v w^+ - w v^+ with p = tau B v,
  // w = p - (tau/2)(v^+ p) v.
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
      for (int i = warp; i < n1; i += kWarps) {
        const double2* brow = A + (k + 1 + i) * lda + (k + 1);
        double2 acc = make_double2(0.0, 0.0);
        for (int j = lane; j < n1; j += 32) c_fma(acc, brow[j], vv[j]);
        acc = warp_all_sum2(acc);
        if (lane == 0) pv[i] = make_double2(tau * acc.x, tau * acc.y);
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

  // Real tridiagonal T_r = P^+ T P with the diagonal phases P_{i+1} = P_i conj(t_i)/|t_i|.
  if (tid == 0) {
    ph[0] = make_double2(1.0, 0.0);
    for (int i = 0; i + 1 < d; ++i) {
      const double2 t = A[i * lda + i + 1];
      const double at = hypot(t.x, t.y);
      ed[i] = at;
      ph[i + 1] = at > 0.0 ? c_mul(ph[i], make_double2(t.x / at, -t.y / at)) : ph[i];
    }
    ed[d - 1] = 0.0;
  }
  for (int i = tid; i < d; i += kT) ad[i] = A[i * lda + i].x;
  for (int idx = tid; idx < d * d; idx += kT) Z[(idx / d) * lda + idx % d] = (idx / d == idx % d) ? 1.0 : 0.0;
  __syncthreads();
  if (warp == 0) tridiagonal_ql(ad, ed, Z, d, lda, p.err);
  __syncthreads();

  // Eigenvectors of H_n: Y = H_0 H_1 ... H_{d-3} P Z, applied right to left.
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, c = idx % d;
    const double z = Z[i * lda + c];
    A[i * lda + c] = make_double2(ph[i].x * z, ph[i].y * z);
  }
  __syncthreads();
  for (int k = d - 3; k >= 0; --k) {
    const double tau = htau[k];
    if (tau == 0.0) continue;
    const int n1 = d - k - 1;
    for (int i = tid; i < n1; i += kT) vv[i] = hv[(size_t)k * d + i];
    __syncthreads();
    for (int c = warp; c < d; c += kWarps) {
      double2 acc = make_double2(0.0, 0.0);
      for (int i = lane; i < n1; i += 32) c_fma_conj(acc, vv[i], A[(k + 1 + i) * lda + c]);
      acc = warp_all_sum2(acc);
      acc.x *= tau;
      acc.y *= tau;
      for (int i = lane; i < n1; i += 32) {
        double2& y = A[(k + 1 + i) * lda + c];
        const double2 t = c_mul(vv[i], acc);
        y.x -= t.x;
        y.y -= t.y;
      }
    }
    __syncthreads();
  }

  // Outputs: eigenvalues, eigenvectors (and their transpose), U_n = Y diag(exp(-i lambda dt)) Y^+.
  double* lam = p.lam + (size_t)step * d;
  double2* V = p.V + (size_t)step * dd;
  double2* Vt = p.Vt + (size_t)step * dd;
  for (int i = tid; i < d; i += kT) {
    lam[i] = ad[i];
    double sn, cs;
    sincos(ad[i] * p.dt, &sn, &cs);
    pv[i] = make_double2(cs, -sn);
  }
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, c = idx % d;
    const double2 y = A[i * lda + c];
    V[idx] = y;
    Vt[(size_t)c * d + i] = y;
  }
  __syncthreads();   // every read of hv is done: the step's slice of U may be overwritten
  double2* U = p.U + (size_t)step * dd;
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, j = idx % d;
    const double2* yi = A + i * lda;
    const double2* yj = A + j * lda;
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 0; l < d; ++l) c_fma(acc, c_mul(yi[l], pv[l]), c_conj(yj[l]));
    U[idx] = acc;
  }
}

// Forward sweep of one column h: psi_s = U_s psi_{s-1}; overlaps and the C2 / C3 accumulations.
__global__ void __launch_bounds__(kT) k_eig_forward(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, h = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double2* cur = reinterpret_cast<double2*>(sm);
  double2* nxt = cur + d;
  double* red = reinterpret_cast<double*>(nxt + d);
  const size_t dd = (size_t)d * d, col = (size_t)h * d, slab = (size_t)p.n * d;
  const double2* tgt = p.target + col;
  for (int i = tid; i < d; i += kT) {
    cur[i] = p.psi0[col + i];
    p.psi_hist[col + i] = cur[i];
  }
  __syncthreads();
  double c2 = 0.0;
  for (int s = 0; s < p.N; ++s) {
    const double2* Us = p.U + (size_t)s * dd;
    double2* hist = p.psi_hist + (size_t)(s + 1) * slab + col;
    for (int i = warp; i < d; i += kWarps) {
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
    __syncthreads();
    if (p.part_g3) {
      double2 g = make_double2(0.0, 0.0);
      for (int i = tid; i < d; i += kT) c_fma_conj(g, tgt[i], nxt[i]);
      g = block_all_sum2(g, red);
      if (tid == 0) p.part_g3[(size_t)h * p.N + s] = g;
    }
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
  double2 g = make_double2(0.0, 0.0);
  for (int i = tid; i < d; i += kT) c_fma_conj(g, tgt[i], cur[i]);
  g = block_all_sum2(g, red);
  const double c2s = block_all_sum2(make_double2(c2, 0.0), red).x;
  if (tid == 0) {
    p.part_g[h] = g;
    p.part_c2[h] = c2s;
  }
}

// Backward sweep of one column h: the combined costate
//   chi_N = -(w_fid g / n^2) phi_T + (w_forbid/(N n)) Omega psi_N - (w_tint/(N n^2)) g_N phi_T,
//   chi_{s-1} = U_s^+ chi_s + (w_forbid/(N n)) Omega psi_{s-1} - (w_tint/(N n^2)) g_{s-1} phi_T.
__global__ void __launch_bounds__(kT) k_eig_backward(EigCtx p) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int d = p.d, h = blockIdx.x, tid = threadIdx.x;
  const int parts = kT / d < 1 ? 1 : kT / d;
  double2* cur = reinterpret_cast<double2*>(sm);
  double2* nxt = cur + d;
  double2* tmp = nxt + d;   // parts x d partial products
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
      cur[i] = ch;
      hist[i] = ch;
    }
  }
  __syncthreads();
  for (int s = p.N; s >= 2; --s) {
    const double2* Us = p.U + (size_t)(s - 1) * dd;
    for (int t = tid; t < parts * d; t += kT) {
      const int i = t % d, q = t / d;
      const int j0 = (int)((int64_t)q * d / parts), j1 = (int)((int64_t)(q + 1) * d / parts);
      double2 acc = make_double2(0.0, 0.0);
      for (int j = j0; j < j1; ++j) c_fma_conj(acc, Us[(size_t)j * d + i], cur[j]);
      tmp[(size_t)q * d + i] = acc;
    }
    __syncthreads();
    const double2* psi = p.psi_hist + (size_t)(s - 1) * slab + col;
    double2* hist = p.chi_hist + (size_t)(s - 1) * slab + col;
    double2 c3 = make_double2(0.0, 0.0);
    if (c3w != 0.0) c3 = make_double2(c3w * p.g3[s - 2].x, c3w * p.g3[s - 2].y);
    for (int i = tid; i < d; i += kT) {
      double2 y = tmp[i];
      for (int q = 1; q < parts; ++q) {
        y.x += tmp[(size_t)q * d + i].x;
        y.y += tmp[(size_t)q * d + i].y;
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
    __syncthreads();
    double2* t = cur;
    cur = nxt;
    nxt = t;
  }
}

__device__ __forceinline__ double2 divided_difference(double li, double lj, double dt) {
  // exp((D_i + D_j)/2) sin(theta)/theta, D = -i lambda dt, theta = (lambda_i - lambda_j) dt / 2
  const double th = 0.5 * (li - lj) * dt;
  const double sinc = fabs(th) < 1e-4 ? 1.0 - th * th * (1.0 / 6.0) : sin(th) / th;
  double sn, cs;
  sincos(0.5 * (li + lj) * dt, &sn, &cs);
  return make_double2(cs * sinc, -sn * sinc);
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
  __syncthreads();
  for (int idx = tid; idx < d * d; idx += kT) {
    const int i = idx / d, j = idx % d;
    double2 m = make_double2(0.0, 0.0);
    for (int h = 0; h < n; ++h) c_fma_conj(m, xc[(size_t)h * d + i], xp[(size_t)h * d + j]);
    Q[i * ldq + j] = c_mul(divided_difference(lam[i], lam[j], p.dt), m);
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
    constexpr int kPer = (kEigMaxDim + 31) / 32;   // entries a = lane + 32 q of T_:b held per lane
    double2 t[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int a = lane + 32 * q;
      double2 acc = make_double2(0.0, 0.0);
      if (a < d)
        for (int i = 0; i < d; ++i) c_fma_conj(acc, Vt[(size_t)i * d + a], c[i]);
      t[q] = acc;
    }
    for (int k = 0; k < K; ++k) {
      const double2* hb = p.Hk + (size_t)k * dd + (size_t)b * d;   // H_k[b][a] = conj(H_k[a][b])
      double im = 0.0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        const int a = lane + 32 * q;
        if (a < d) {
          const double2 hba = hb[a];
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
size_t backward_smem(int d) {
  const int parts = kT / d < 1 ? 1 : kT / d;
  return (size_t)16 * (2 + parts) * d;
}

}  // namespace

int eig_step_smem(int d) { return (int)step_layout(d).bytes; }

int eig_grad_smem(int d, int K) {
  return (int)((size_t)16 * d * (d + 1) + (size_t)16 * kWarps * d + (size_t)8 * kWarps * (K > 0 ? K : 1));
}

cudaError_t eig_prepare(int d, int K) {
  cudaError_t e = cudaFuncSetAttribute(k_eig_step, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_step_smem(d));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_eig_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, eig_grad_smem(d, K));
  return e;
}

cudaError_t eig_forward(const EigCtx& c, cudaStream_t st) {
  k_eig_step<<<c.N, kT, eig_step_smem(c.d), st>>>(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_eig_forward<<<c.n, kT, forward_smem(c.d), st>>>(c);
  return cudaGetLastError();
}

cudaError_t eig_backward(const EigCtx& c, cudaStream_t st) {
  k_eig_backward<<<c.n, kT, backward_smem(c.d), st>>>(c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || c.K == 0) return e;
  k_eig_grad<<<c.N, kT, eig_grad_smem(c.d, c.K), st>>>(c);
  return cudaGetLastError();
}

}  // namespace grape
