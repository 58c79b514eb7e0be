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
// barrier (__syncthreads for CL = 1, barrier.cluster otherwise).  Nothing is
// exchanged through global memory inside a sweep.
//
// Kernels
//   k_schedule      ||A_n||_1 = dt max_i sum_j |H_n,ij| and the (m_n, s_n) lookup (Sec. III.B, App. C)
//   k_forward       psi_n = (e^{B_n}_m)^s psi_{n-1}, C2 sum, checkpoints, psi_N, <phi_T|psi_N> partials
//   k_finalize      g, C1, C2, C_amp, cost
//   k_backward      adjoint re-propagation of psi and the costate, gradient terms per step
//   k_grad_reduce   sum of per-CTA gradient partials + amplitude-penalty gradient
#include "grape_internal.h"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace grape {

// 1/q and 1/q! for q = 0..kMaxTaylor
__constant__ double c_inv_int[kMaxTaylor + 2];
__constant__ double c_inv_fact[kMaxTaylor + 2];

static bool g_constants_ready[64] = {false};

static cudaError_t ensure_constants() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && g_constants_ready[dev]) return cudaSuccess;
  double inv_int[kMaxTaylor + 2], inv_fact[kMaxTaylor + 2];
  inv_int[0] = 0.0;
  inv_fact[0] = 1.0;
  for (int q = 1; q < kMaxTaylor + 2; ++q) {
    inv_int[q] = 1.0 / q;
    inv_fact[q] = inv_fact[q - 1] / q;
  }
  e = cudaMemcpyToSymbol(c_inv_int, inv_int, sizeof(inv_int));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_inv_fact, inv_fact, sizeof(inv_fact));
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

// One block per step (grid-strided).  ||A_n||_1 = dt * max_i sum_j |H_n,ij| on the union pattern
// (the 1-norm equals the infinity norm for Hermitian H, footnote to Eq. (norm inequality)).
__global__ void __launch_bounds__(256) k_schedule(ScheduleParams p) {
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  for (int n = blockIdx.x; n < p.N; n += gridDim.x) {
    __syncthreads();
    if (threadIdx.x < p.K) s_u[threadIdx.x] = p.u[(int64_t)threadIdx.x * p.N + n];
    __syncthreads();
    double rmax = 0.0;
    bool bad = false;
    for (int i = threadIdx.x; i < p.dim; i += blockDim.x) {
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
    if (bad) rmax = __longlong_as_double(0x7ff0000000000000LL);   // +inf marks a non-finite step
    const double mx = block_max(rmax, red);
    if (threadIdx.x == 0) {
      const double x = p.dt * mx;
      int m = 0, s = 0;
      if (!(x <= 1e300)) {
        set_error(p.err, kErrNonFinite);
      } else {
        for (int si = 1; si <= p.s_cap && s == 0; ++si) {
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
  }
}

// ------------------------------------------------------------------ sweep helpers

struct Carve {
  double2* xb;        // exchange buffers (local)
  double2* psi;
  double2* chi;
  double2* inc;
  double2* vals;
  double2* W;
  double2* wsm;       // Horner slots in shared memory (first m_smem)
  double2* wgl;       // Horner slots in global scratch (slots >= m_smem)
  int* lrow;
  uint32_t* lcol;
};

__device__ __forceinline__ Carve carve(unsigned char* smem, const SweepParams& p, bool backward, int part) {
  const SmemLayout L = make_layout(backward, p.R, p.max_nnz_loc, p.in_smem, p.m_smem, 16);
  double2* scr = p.scratch + (int64_t)part * p.scratch_stride;
  Carve c;
  c.xb = reinterpret_cast<double2*>(smem + L.xbuf);
  c.psi = reinterpret_cast<double2*>(smem + L.psi);
  c.chi = backward ? reinterpret_cast<double2*>(smem + L.chi) : nullptr;
  c.inc = reinterpret_cast<double2*>(smem + L.inc);
  c.vals = L.vals >= 0 ? reinterpret_cast<double2*>(smem + L.vals) : scr + p.scr_vals;
  c.W = L.W >= 0 ? reinterpret_cast<double2*>(smem + L.W) : scr + p.scr_W;
  c.wsm = L.wslot >= 0 ? reinterpret_cast<double2*>(smem + L.wslot) : nullptr;
  c.wgl = scr + p.scr_wslot;
  c.lrow = reinterpret_cast<int*>(smem + L.lrow);
  c.lcol = reinterpret_cast<uint32_t*>(smem + L.lcol);
  return c;
}

// Horner slot p of local row i.
__device__ __forceinline__ double2* wslot_ptr(const Carve& c, int m_smem, int R, int p, int i) {
  return p < m_smem ? c.wsm + (int64_t)p * R + i : c.wgl + (int64_t)(p - m_smem) * R + i;
}

// Table of generic pointers to exchange buffer `b` of every CTA of the team.
template <bool CLUSTER>
struct XTab {
  double2* ptr[kMaxCluster];
};

// Assemble B_n = -i dt H_n / s on the CTA's local entries: vals[e] = (dt/s) * (-i) * (h0 + sum_k u_kn h_k).
__device__ __forceinline__ void assemble(const SweepParams& p, const Carve& c, int64_t e0, int nnz_loc, int n,
                                         double scale, const double* s_u) {
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) {
    const int64_t ge = e0 + e;
    double2 v = p.h0v[ge];
    for (int k = p.ectr_ptr[ge]; k < p.ectr_ptr[ge + 1]; ++k) {
      const double uk = s_u[p.ectr_k[k]];
      const double2 hv = p.ectr_val[k];
      v.x = fma(uk, hv.x, v.x);
      v.y = fma(uk, hv.y, v.y);
    }
    c.vals[e] = make_double2(scale * v.y, -scale * v.x);   // -i v
  }
}

__device__ __forceinline__ void load_controls(const SweepParams& p, int n, double* s_u) {
  if (threadIdx.x < p.K) s_u[threadIdx.x] = p.u[(int64_t)threadIdx.x * p.N + n];
}

template <bool CLUSTER>
__device__ __forceinline__ double2 xload(const double2* local, const XTab<CLUSTER>& tab, uint32_t enc) {
  if constexpr (CLUSTER) {
    return tab.ptr[(enc >> kOwnerShift) & 0xFFu][enc & kLocalMask];
  } else {
    return local[enc & kLocalMask];
  }
}

template <bool CLUSTER>
__device__ __forceinline__ void sweep_setup(const SweepParams& p, const Carve& c, int r0, int nrows, int64_t e0,
                                            int nnz_loc) {
  for (int i = threadIdx.x; i <= nrows; i += blockDim.x) c.lrow[i] = (int)(p.rowptr[r0 + i] - e0);
  for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) c.lcol[e] = p.colenc[e0 + e];
}

// ------------------------------------------------------------------ forward sweep

// psi_n = (e^{B}_m)^s psi_{n-1} by the recursions b_j = (B/j) b_{j-1} (App. C Eq. (recursive relation 1))
// and c_l = e^B_m c_{l-1} (Eq. (recursive relation2)); C2 accumulates <psi_n|Omega|psi_n> (App. A).
template <bool CLUSTER>
__global__ void __launch_bounds__(1024, 1) k_forward(SweepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<CLUSTER> tab[2];
  const int part = blockIdx.x;
  const int team = part / p.CL, rank = part % p.CL;
  const int r0 = min(rank * p.R, p.dim), r1 = min(r0 + p.R, p.dim), nrows = r1 - r0;
  const int64_t e0 = p.rowptr[r0];
  const int nnz_loc = (int)(p.rowptr[r1] - e0);
  const Carve c = carve(smem, p, false, part);
  double2* T[2] = {c.xb, c.xb + p.R};
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL) {
      tab[0].ptr[threadIdx.x] = cl.map_shared_rank(T[0], threadIdx.x);
      tab[1].ptr[threadIdx.x] = cl.map_shared_rank(T[1], threadIdx.x);
    }
  }
  sweep_setup<CLUSTER>(p, c, r0, nrows, e0, nnz_loc);
  const int64_t col0 = (int64_t)team * p.dim + r0;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) c.psi[i] = p.psi0[col0 + i];
  double c2acc = 0.0;
  team_sync<CLUSTER>();
  for (int n = 0; n < p.N; ++n) {
    const int m = p.ms_m[n], s = p.ms_s[n];
    if (s <= 0 || m <= 0) continue;   // flagged by k_schedule; uniform over the team
    load_controls(p, n, s_u);
    __syncthreads();
    assemble(p, c, e0, nnz_loc, n, p.dt / s, s_u);
    __syncthreads();
    for (int l = 0; l < s; ++l) {
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        T[0][i] = c.psi[i];
        c.inc[i] = make_double2(0.0, 0.0);
      }
      team_sync<CLUSTER>();
      for (int q = 1; q <= m; ++q) {
        const int src = (q - 1) & 1, dst = q & 1;
        const double iq = c_inv_int[q];
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          double2 y = make_double2(0.0, 0.0);
          const int ea = c.lrow[i], eb = c.lrow[i + 1];
          for (int e = ea; e < eb; ++e) cmac(y, c.vals[e], xload<CLUSTER>(T[src], tab[src], c.lcol[e]));
          y = cscale(y, iq);
          T[dst][i] = y;
          double2 a = c.inc[i];
          a.x += y.x;
          a.y += y.y;
          c.inc[i] = a;
        }
        team_sync<CLUSTER>();
      }
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        double2 v = c.psi[i];
        const double2 a = c.inc[i];
        v.x += a.x;
        v.y += a.y;
        c.psi[i] = v;
      }
    }
    // psi now holds psi_{n+1}
    if (p.omega) {
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        const double2 v = c.psi[i];
        c2acc = fma(p.omega[r0 + i], v.x * v.x + v.y * v.y, c2acc);
      }
    }
    if (p.ckpt_every > 0 && (n + 1) % p.ckpt_every == 0) {
      const int slot = (n + 1) / p.ckpt_every - 1;
      if (slot < p.n_ckpt) {
        double2* dst = p.ckpt + ((int64_t)slot * p.n_states + team) * p.dim + r0;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) dst[i] = c.psi[i];
      }
    }
  }
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
  team_sync<CLUSTER>();   // no CTA leaves while a team member may still read its shared memory
}

// ------------------------------------------------------------------ finalize (one block)

__global__ void __launch_bounds__(256) k_finalize(FinalizeParams p) {
  __shared__ double red[32];
  double gx = 0.0, gy = 0.0, c2 = 0.0, a2 = 0.0;
  for (int i = threadIdx.x; i < p.n_parts; i += blockDim.x) {
    gx += p.part_g[i].x;
    gy += p.part_g[i].y;
    c2 += p.part_c2[i];
  }
  for (int64_t i = threadIdx.x; i < (int64_t)p.K * p.N; i += blockDim.x) a2 = fma(p.u[i], p.u[i], a2);
  gx = block_sum(gx, red);
  gy = block_sum(gy, red);
  c2 = block_sum(c2, red);
  a2 = block_sum(a2, red);
  if (threadIdx.x == 0) {
    const double n = (double)p.n_states;
    const double C1 = 1.0 - (gx * gx + gy * gy) / (n * n);
    const double C2 = c2 / ((double)p.N * n);
    const double Ca = a2 / (double)p.N;
    *p.g_out = make_double2(gx, gy);
    *p.cost_out = p.w_fid * C1 + p.w_forbid * C2 + p.w_amp * Ca;
    if (p.parts_out) {
      p.parts_out[0] = C1;
      p.parts_out[1] = C2;
      p.parts_out[2] = Ca;
      p.parts_out[3] = sqrt(gx * gx + gy * gy);
    }
  }
}

// ------------------------------------------------------------------ backward sweep

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
template <bool CLUSTER>
__global__ void __launch_bounds__(1024, 1) k_backward(SweepParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ double s_u[kMaxControls];
  __shared__ XTab<CLUSTER> tab[6];
  const int part = blockIdx.x;
  const int team = part / p.CL, rank = part % p.CL;
  const int r0 = min(rank * p.R, p.dim), r1 = min(r0 + p.R, p.dim), nrows = r1 - r0;
  const int64_t e0 = p.rowptr[r0];
  const int nnz_loc = (int)(p.rowptr[r1] - e0);
  const Carve c = carve(smem, p, true, part);
  const int R = p.R;
  // exchange buffers: A (psi chain) 0,1; W (Horner chain) 2,3; X (x chain) 4,5
  double2* X[6] = {c.xb, c.xb + R, c.xb + 2 * R, c.xb + 3 * R, c.xb + 4 * R, c.xb + 5 * R};
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x < p.CL)
      for (int b = 0; b < 6; ++b) tab[b].ptr[threadIdx.x] = cl.map_shared_rank(X[b], threadIdx.x);
  }
  sweep_setup<CLUSTER>(p, c, r0, nrows, e0, nnz_loc);
  const int64_t col0 = (int64_t)team * p.dim + r0;
  const double nS = (double)p.n_states;
  const double2 g = *p.g_final;
  const double2 coefA = make_double2(-p.w_fid * g.x / (nS * nS), -p.w_fid * g.y / (nS * nS));
  const double c2w = (p.omega && p.w_forbid != 0.0) ? p.w_forbid / ((double)p.N * nS) : 0.0;
  for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
    const double2 v = p.psiN[col0 + i];
    c.psi[i] = v;
    double2 ch = cmul(coefA, p.target[col0 + i]);
    if (c2w != 0.0) {
      const double w = c2w * p.omega[r0 + i];
      ch.x = fma(w, v.x, ch.x);
      ch.y = fma(w, v.y, ch.y);
    }
    c.chi[i] = ch;
  }
  team_sync<CLUSTER>();
  for (int n = p.N - 1; n >= 0; --n) {
    const int m = p.ms_m[n], s = p.ms_s[n];
    if (s <= 0 || m <= 0) continue;
    load_controls(p, n, s_u);
    __syncthreads();
    assemble(p, c, e0, nnz_loc, n, p.dt / s, s_u);
    for (int e = threadIdx.x; e < nnz_loc; e += blockDim.x) c.W[e] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int l = s - 1; l >= 0; --l) {
      // ---------------- phase A: psi and Horner chains with -B
      const double fm = c_inv_fact[m];
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        X[0][i] = c.psi[i];
        c.inc[i] = make_double2(0.0, 0.0);
        const double2 w0 = cscale(c.chi[i], fm);
        X[2][i] = w0;
        *wslot_ptr(c, p.m_smem, R, m - 1, i) = w0;
      }
      team_sync<CLUSTER>();
      for (int q = 1; q <= m; ++q) {
        const int src = (q - 1) & 1, dst = q & 1;
        const double iq = c_inv_int[q];
        const double fq = c_inv_fact[m - q];
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          double2 ya = make_double2(0.0, 0.0), yw = make_double2(0.0, 0.0);
          const int ea = c.lrow[i], eb = c.lrow[i + 1];
          for (int e = ea; e < eb; ++e) {
            const uint32_t enc = c.lcol[e];
            const double2 v = c.vals[e];
            cmac(ya, v, xload<CLUSTER>(X[src], tab[src], enc));
            cmac(yw, v, xload<CLUSTER>(X[2 + src], tab[2 + src], enc));
          }
          ya = cscale(ya, -iq);                       // (-B) a_{q-1} / q
          X[dst][i] = ya;
          double2 a = c.inc[i];
          a.x += ya.x;
          a.y += ya.y;
          c.inc[i] = a;
          const double2 ch = c.chi[i];
          const double2 w = make_double2(fma(ch.x, fq, -yw.x), fma(ch.y, fq, -yw.y));   // chi/(p+1)! + (-B) w_{p+1}
          X[2 + dst][i] = w;
          if (q < m) *wslot_ptr(c, p.m_smem, R, m - 1 - q, i) = w;
          else c.chi[i] = w;                           // chi^(l) = w_{-1}
        }
        team_sync<CLUSTER>();
      }
      // ---------------- phase B: x chain with B, accumulate W on control entries
      for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
        double2 v = c.psi[i];
        const double2 a = c.inc[i];
        v.x += a.x;
        v.y += a.y;
        c.psi[i] = v;                                  // psi^(l)
        X[4][i] = v;
      }
      team_sync<CLUSTER>();
      for (int pp = 0; pp < m; ++pp) {
        const int src = pp & 1, dst = src ^ 1;
        const bool more = pp < m - 1;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          const double2 wp = *wslot_ptr(c, p.m_smem, R, pp, i);
          double2 y = make_double2(0.0, 0.0);
          const int ea = c.lrow[i], eb = c.lrow[i + 1];
          for (int e = ea; e < eb; ++e) {
            const uint32_t enc = c.lcol[e];
            const double2 x = xload<CLUSTER>(X[4 + src], tab[4 + src], enc);
            if (more) cmac(y, c.vals[e], x);
            if (enc & kCtrlBit) {
              double2 acc = c.W[e];
              cmac_conj(acc, wp, x);
              c.W[e] = acc;
            }
          }
          if (more) X[4 + dst][i] = y;
        }
        if (more) team_sync<CLUSTER>();
      }
    }
    // ---------------- step end: psi ~ psi_n (0-based state index n), costate source, gradient
    __syncthreads();
    if (n > 0) {
      if (p.ckpt_every > 0 && n % p.ckpt_every == 0 && n / p.ckpt_every - 1 < p.n_ckpt) {
        const double2* srcp = p.ckpt + ((int64_t)(n / p.ckpt_every - 1) * p.n_states + team) * p.dim + r0;
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) c.psi[i] = srcp[i];
      }
      if (c2w != 0.0) {
        for (int i = threadIdx.x; i < nrows; i += blockDim.x) {
          const double w = c2w * p.omega[r0 + i];
          const double2 v = c.psi[i];
          double2 ch = c.chi[i];
          ch.x = fma(w, v.x, ch.x);
          ch.y = fma(w, v.y, ch.y);
          c.chi[i] = ch;
        }
      }
    }
    // dC/du_kn part = 2 Re sum_ij (C_k)_ij W_ij, C_k = -i (dt/s) h_k: Re(-i h W) = h.x W.y + h.y W.x
    const double gscale = 2.0 * p.dt / s;
    for (int k = 0; k < p.K; ++k) {
      const int lo = p.cslice[(k * p.CL + rank) * 2], hi = p.cslice[(k * p.CL + rank) * 2 + 1];
      double acc = 0.0;
      for (int cc = lo + threadIdx.x; cc < hi; cc += blockDim.x) {
        const int e = (int)(p.cidx[cc] - e0);
        const double2 w = c.W[e];
        const double2 h = p.cval[cc];
        acc = fma(h.x, w.y, acc);
        acc = fma(h.y, w.x, acc);
      }
      const double tot = block_sum(acc, red);
      if (threadIdx.x == 0) p.part_grad[((int64_t)part * p.N + n) * p.K + k] = gscale * tot;
    }
    __syncthreads();
  }
  team_sync<CLUSTER>();
}

// ------------------------------------------------------------------ gradient reduce

__global__ void k_grad_reduce(GradReduceParams p) {
  const int64_t total = (int64_t)p.K * p.N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / p.N), n = (int)(idx % p.N);
    double acc = 0.0;
    for (int part = 0; part < p.n_parts; ++part) acc += p.part_grad[((int64_t)part * p.N + n) * p.K + k];
    p.grad[idx] = acc + p.w_amp * 2.0 * p.u[idx] / (double)p.N;
  }
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
  const int grid = p.N < 1216 ? p.N : 1216;
  k_schedule<<<grid, 256, 0, st>>>(p);
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
  (void)precision;
  if (p.CL > 1) return launch_sweep(k_forward<true>, p, smem_bytes, threads, st);
  return launch_sweep(k_forward<false>, p, smem_bytes, threads, st);
}

cudaError_t launch_backward(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st) {
  (void)precision;
  if (p.CL > 1) return launch_sweep(k_backward<true>, p, smem_bytes, threads, st);
  return launch_sweep(k_backward<false>, p, smem_bytes, threads, st);
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

cudaError_t check_nonfinite_u(const double* u, int64_t count, int* err, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int grid = (int)((count + 255) / 256);
  if (grid > 1024) grid = 1024;
  k_check_finite<<<grid, 256, 0, st>>>(u, count, err);
  return cudaGetLastError();
}

}  // namespace grape
