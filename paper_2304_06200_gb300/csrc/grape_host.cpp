// C ABI of the HG GRAPE library: validation, union sparsity pattern, (m, s) table,
// device memory plan and the launch sequence of one evaluation.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <limits>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/grape_hg.h"
#include "grape_bound.h"
#include "grape_internal.h"

using cplx = std::complex<double>;

namespace {

thread_local std::string g_last_error;

grape_status fail(grape_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

grape_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return GRAPE_ECUDA;
}

// Makes `dev` current for the scope of an ABI call and restores the caller's device.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct HostCSR {
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<cplx> val;
};

grape_status to_csr(const grape_op& op, int64_t dim, const char* name, HostCSR& out) {
  out.rowptr.assign(dim + 1, 0);
  out.col.clear();
  out.val.clear();
  if (op.fmt == GRAPE_DENSE) {
    if (!op.values) return fail(GRAPE_EINVAL, std::string(name) + ": dense values pointer is NULL");
    for (int64_t i = 0; i < dim; ++i) {
      for (int64_t j = 0; j < dim; ++j) {
        const double re = op.values[2 * (i * dim + j)], im = op.values[2 * (i * dim + j) + 1];
        if (!std::isfinite(re) || !std::isfinite(im)) return fail(GRAPE_EINVAL, std::string(name) + ": non-finite entry");
        if (re != 0.0 || im != 0.0) {
          out.col.push_back((int32_t)j);
          out.val.emplace_back(re, im);
        }
      }
      out.rowptr[i + 1] = (int64_t)out.col.size();
    }
    return GRAPE_OK;
  }
  if (op.fmt != GRAPE_CSR) return fail(GRAPE_EINVAL, std::string(name) + ": unknown format");
  if (op.nnz < 0) return fail(GRAPE_EINVAL, std::string(name) + ": negative nnz");
  if (op.nnz > 0 && (!op.rowptr || !op.colind || !op.values))
    return fail(GRAPE_EINVAL, std::string(name) + ": CSR pointer is NULL");
  if (op.nnz == 0 && !op.rowptr) {
    return GRAPE_OK;   // empty operator
  }
  if (op.rowptr[0] != 0 || op.rowptr[dim] != op.nnz) return fail(GRAPE_EINVAL, std::string(name) + ": bad rowptr ends");
  std::vector<std::pair<int32_t, cplx>> row;
  for (int64_t i = 0; i < dim; ++i) {
    const int64_t a = op.rowptr[i], b = op.rowptr[i + 1];
    if (b < a || b > op.nnz) return fail(GRAPE_EINVAL, std::string(name) + ": rowptr not monotone");
    row.clear();
    for (int64_t e = a; e < b; ++e) {
      const int32_t j = op.colind[e];
      if (j < 0 || j >= dim) return fail(GRAPE_EINVAL, std::string(name) + ": column index out of range");
      const double re = op.values[2 * e], im = op.values[2 * e + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) return fail(GRAPE_EINVAL, std::string(name) + ": non-finite entry");
      row.emplace_back(j, cplx(re, im));
    }
    std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    for (size_t t = 0; t < row.size(); ++t) {
      if (t > 0 && row[t].first == row[t - 1].first)
        return fail(GRAPE_EINVAL, std::string(name) + ": duplicate entry in a row");
      if (row[t].second == cplx(0.0, 0.0)) continue;
      out.col.push_back(row[t].first);
      out.val.push_back(row[t].second);
    }
    out.rowptr[i + 1] = (int64_t)out.col.size();
  }
  return GRAPE_OK;
}

bool lookup(const HostCSR& A, int64_t i, int32_t j, cplx* v) {
  const auto b = A.col.begin() + A.rowptr[i], e = A.col.begin() + A.rowptr[i + 1];
  const auto it = std::lower_bound(b, e, j);
  if (it == e || *it != j) return false;
  *v = A.val[it - A.col.begin()];
  return true;
}

bool is_hermitian(const HostCSR& A, int64_t dim) {
  double scale = 0.0;
  for (const auto& v : A.val) scale = std::max(scale, std::abs(v));
  const double tol = 1e-12 * std::max(scale, 1e-300);
  for (int64_t i = 0; i < dim; ++i) {
    for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) {
      const int32_t j = A.col[e];
      cplx t(0.0, 0.0);
      lookup(A, j, (int32_t)i, &t);
      if (std::abs(A.val[e] - std::conj(t)) > tol) return false;
    }
  }
  return true;
}

}  // namespace

namespace grape {
// Lets other translation units of the library report a message through grape_last_error().
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace grape

struct grape_problem {
  int device = 0;
  int64_t dim = 0;
  int K = 0, N = 0, n = 0;
  double dt = 0, w_fid = 0, w_forbid = 0, w_amp = 0, tau = 0;
  int precision = 0, CL = 1, R = 0, ckpt_every = 0, n_ckpt = 0, m_cap = 0, s_cap = 0, sigma = 0;
  int64_t nnz = 0, n_ctr = 0;
  bool has_omega = false;
  grape_alloc_fn alloc_fn = nullptr;
  grape_free_fn free_fn = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<std::pair<void*, size_t>> allocations;
  int64_t device_bytes = 0;
  grape::ScheduleTable table;
  // device buffers
  int64_t* d_rowptr = nullptr;
  uint32_t* d_colenc = nullptr;
  double2* d_h0v = nullptr;
  int* d_cptr = nullptr;
  int* d_cidx = nullptr;
  double2* d_cval = nullptr;
  int* d_cslice = nullptr;
  int* d_ectr_ptr = nullptr;
  int* d_ectr_k = nullptr;
  double2* d_ectr_val = nullptr;
  double* d_table = nullptr;
  double* d_table_smax = nullptr;
  double2* d_psi0 = nullptr;
  double2* d_target = nullptr;
  double* d_omega = nullptr;
  double* d_u = nullptr;
  int* d_ms_m = nullptr;
  int* d_ms_s = nullptr;
  double* d_norm1 = nullptr;
  double2* d_psiN = nullptr;
  double2* d_ckpt = nullptr;
  double2* d_part_g = nullptr;
  double* d_part_c2 = nullptr;
  double* d_part_grad = nullptr;
  double2* d_g = nullptr;
  double* d_cost = nullptr;
  double* d_parts = nullptr;
  double* d_grad = nullptr;
  double2* d_scratch = nullptr;
  int* d_err = nullptr;
  // launch plan
  int threads = 0, fwd_smem = 0, bwd_smem = 0, fwd_in_smem = 0, bwd_in_smem = 0, m_smem = 0, max_nnz_loc = 0;
  int64_t scratch_stride = 0, scr_vals = 0, scr_W = 0, scr_wslot = 0;
  bool forward_done = false;
  bool evaluated = false;
  cudaStream_t last_stream = nullptr;

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (alloc_fn) {
      p = alloc_fn(bytes, alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) {
      allocations.emplace_back(p, bytes);
      device_bytes += (int64_t)bytes;
    }
    return p;
  }
  void release() {
    for (auto& a : allocations) {
      if (free_fn) free_fn(a.first, a.second, alloc_ctx);
      else cudaFree(a.first);
    }
    allocations.clear();
    device_bytes = 0;
  }
};

namespace {

template <typename T>
grape_status upload(grape_problem* P, T** dst, const T* src, size_t count) {
  *dst = static_cast<T*>(P->dalloc(count * sizeof(T)));
  if (!*dst) return fail(GRAPE_ENOMEM, "device allocation failed");
  if (count && src) {
    cudaError_t e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (upload)");
  }
  return GRAPE_OK;
}

template <typename T>
grape_status dzeros(grape_problem* P, T** dst, size_t count) {
  *dst = static_cast<T*>(P->dalloc(count * sizeof(T)));
  if (!*dst) return fail(GRAPE_ENOMEM, "device allocation failed");
  cudaError_t e = cudaMemset(*dst, 0, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  return GRAPE_OK;
}

int sm_count(int dev) {
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return std::max(v, 1);
}

grape_status build(grape_problem* P, const grape_desc* d) {
  const int64_t dim = d->dim;
  const int K = d->n_controls;
  // ---- operators on the host
  std::vector<HostCSR> ops(K + 1);
  grape_status st = to_csr(d->H0, dim, "H0", ops[0]);
  if (st) return st;
  for (int k = 0; k < K; ++k) {
    const std::string nm = "H_" + std::to_string(k);
    st = to_csr(d->Hk[k], dim, nm.c_str(), ops[k + 1]);
    if (st) return st;
  }
  for (int k = 0; k <= K; ++k)
    if (!is_hermitian(ops[k], dim))
      return fail(GRAPE_ENOTHERMITIAN, k == 0 ? "H0 is not Hermitian" : "H_" + std::to_string(k - 1) + " is not Hermitian");
  // ---- union pattern
  std::vector<int64_t> rowptr(dim + 1, 0);
  std::vector<int32_t> ucol;
  std::vector<int32_t> rowbuf;
  for (int64_t i = 0; i < dim; ++i) {
    rowbuf.clear();
    for (int k = 0; k <= K; ++k)
      for (int64_t e = ops[k].rowptr[i]; e < ops[k].rowptr[i + 1]; ++e) rowbuf.push_back(ops[k].col[e]);
    std::sort(rowbuf.begin(), rowbuf.end());
    rowbuf.erase(std::unique(rowbuf.begin(), rowbuf.end()), rowbuf.end());
    ucol.insert(ucol.end(), rowbuf.begin(), rowbuf.end());
    rowptr[i + 1] = (int64_t)ucol.size();
  }
  const int64_t nnz = (int64_t)ucol.size();
  if (nnz >= (int64_t)std::numeric_limits<int>::max()) return fail(GRAPE_EINVAL, "union pattern too large");
  P->nnz = nnz;
  int sigma = 0;
  for (int64_t i = 0; i < dim; ++i) sigma = std::max<int>(sigma, (int)(rowptr[i + 1] - rowptr[i]));
  P->sigma = std::max(sigma, 1);
  auto uindex = [&](int64_t i, int32_t j) -> int64_t {
    const auto b = ucol.begin() + rowptr[i], e = ucol.begin() + rowptr[i + 1];
    return (int64_t)(std::lower_bound(b, e, j) - ucol.begin());
  };
  std::vector<double2> h0v(nnz, make_double2(0.0, 0.0));
  for (int64_t i = 0; i < dim; ++i)
    for (int64_t e = ops[0].rowptr[i]; e < ops[0].rowptr[i + 1]; ++e) {
      const cplx v = ops[0].val[e];
      h0v[uindex(i, ops[0].col[e])] = make_double2(v.real(), v.imag());
    }
  // per-control lists (sorted by union entry) and entry-major lists
  std::vector<int> cptr(K + 1, 0), cidx;
  std::vector<double2> cval;
  std::vector<std::vector<std::pair<int, double2>>> per_entry(nnz);
  for (int k = 0; k < K; ++k) {
    for (int64_t i = 0; i < dim; ++i)
      for (int64_t e = ops[k + 1].rowptr[i]; e < ops[k + 1].rowptr[i + 1]; ++e) {
        const int64_t ue = uindex(i, ops[k + 1].col[e]);
        const cplx v = ops[k + 1].val[e];
        cidx.push_back((int)ue);
        cval.push_back(make_double2(v.real(), v.imag()));
        per_entry[ue].emplace_back(k, make_double2(v.real(), v.imag()));
      }
    cptr[k + 1] = (int)cidx.size();
  }
  P->n_ctr = (int64_t)cidx.size();
  std::vector<int> ectr_ptr(nnz + 1, 0), ectr_k;
  std::vector<double2> ectr_val;
  for (int64_t e = 0; e < nnz; ++e) {
    for (auto& pr : per_entry[e]) {
      ectr_k.push_back(pr.first);
      ectr_val.push_back(pr.second);
    }
    ectr_ptr[e + 1] = (int)ectr_k.size();
  }
  // ---- (m, s) breakpoint table (App. C)
  const double uround = grape::unit_roundoff(P->precision);
  P->table = grape::build_table(P->tau, P->sigma, uround, P->m_cap, 4096, 2000.0);
  if (P->table.x_max < 0.0) return fail(GRAPE_ETOL, "no (m, s) pair satisfies E_A <= tau even for ||A||_1 = 0");
  P->m_cap = P->table.m_cap;
  P->s_cap = P->table.s_cap;
  // ---- team size: CTAs per column (cost model: FP64 lanes per SM per clock ~1.7, team barrier
  // ~80 clocks inside one CTA and ~1100 clocks (barrier + remote read latency) across a cluster)
  const int dev = P->device;
  const int nsm = sm_count(dev);
  const int smem_max = grape::max_dynamic_smem(dev) - 2048;   // static shared memory of the kernels
  auto plan_for = [&](int CL, int* R_out, int* mnl_out) -> bool {
    const int64_t R = (dim + CL - 1) / CL;
    if (R >= (1 << 20)) return false;
    int mnl = 0;
    for (int r = 0; r < CL; ++r) {
      const int64_t r0 = std::min<int64_t>((int64_t)r * R, dim), r1 = std::min<int64_t>(r0 + R, dim);
      mnl = std::max<int>(mnl, (int)(rowptr[r1] - rowptr[r0]));
    }
    const int fixed = grape::make_layout(true, (int)R, mnl, 0, 0, 16).total;
    if (fixed > smem_max) return false;
    *R_out = (int)R;
    *mnl_out = mnl;
    return true;
  };
  int bestCL = 0, bestR = 0, bestMnl = 0;
  double bestCost = 1e300;
  const int cands[5] = {1, 2, 4, 8, 16};
  for (int ci = 0; ci < 5; ++ci) {
    const int CL = cands[ci];
    if (d->cluster > 0 && CL != d->cluster) continue;
    if (CL > 1 && CL > dim) continue;
    int R = 0, mnl = 0;
    if (!plan_for(CL, &R, &mnl)) continue;
    const double work = mnl * 4.0 / 1.7;
    const double sync = CL == 1 ? 80.0 : 1100.0;
    const double waves = std::ceil((double)d->n_states * CL / nsm);
    const double cost = waves * (work + sync);
    if (cost < bestCost * 0.98) {
      bestCost = cost;
      bestCL = CL;
      bestR = R;
      bestMnl = mnl;
    }
  }
  if (bestCL == 0) return fail(GRAPE_EINVAL, "problem does not fit the sweep kernels' shared memory for any team size");
  P->CL = bestCL;
  P->R = bestR;
  P->max_nnz_loc = std::max(bestMnl, 1);
  const int CL = P->CL, R = P->R;
  // column encoding for this partition
  std::vector<uint32_t> colenc(nnz);
  for (int64_t i = 0; i < dim; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int32_t j = ucol[e];
      const uint32_t owner = (uint32_t)(j / R), local = (uint32_t)(j - (int64_t)owner * R);
      uint32_t enc = (owner << grape::kOwnerShift) | local;
      if (ectr_ptr[e + 1] > ectr_ptr[e]) enc |= grape::kCtrlBit;
      colenc[e] = enc;
    }
  std::vector<int> cslice((size_t)std::max(K, 1) * CL * 2, 0);
  for (int k = 0; k < K; ++k)
    for (int r = 0; r < CL; ++r) {
      const int64_t r0 = std::min<int64_t>((int64_t)r * R, dim), r1 = std::min<int64_t>(r0 + R, dim);
      const auto b = cidx.begin() + cptr[k], e = cidx.begin() + cptr[k + 1];
      cslice[(k * CL + r) * 2] = (int)(std::lower_bound(b, e, (int)rowptr[r0]) - cidx.begin());
      cslice[(k * CL + r) * 2 + 1] = (int)(std::lower_bound(b, e, (int)rowptr[r1]) - cidx.begin());
    }
  // ---- shared-memory plan
  const int mnl = P->max_nnz_loc;
  int fin = 0;
  if (grape::make_layout(false, R, mnl, 1, 0, 16).total <= smem_max) fin = 1;
  P->fwd_in_smem = fin;
  P->fwd_smem = grape::make_layout(false, R, mnl, fin, 0, 16).total;
  int bin = 0;
  if (grape::make_layout(true, R, mnl, 1, 0, 16).total <= smem_max) bin = 1;
  if (grape::make_layout(true, R, mnl, bin | 2, 0, 16).total <= smem_max) bin |= 2;
  const int base = grape::make_layout(true, R, mnl, bin, 0, 16).total;
  int m_smem = (int)std::min<int64_t>(P->m_cap, (smem_max - base - 16) / std::max<int64_t>((int64_t)R * 16, 1));
  m_smem = std::max(m_smem, 0);
  P->bwd_in_smem = bin;
  P->m_smem = m_smem;
  P->bwd_smem = grape::make_layout(true, R, mnl, bin, m_smem, 16).total;
  P->threads = (int)std::min<int64_t>(1024, std::max<int64_t>(64, ((int64_t)R + 31) / 32 * 32));
  P->scr_vals = 0;
  P->scr_W = mnl;
  P->scr_wslot = 2 * (int64_t)mnl;
  P->scratch_stride = 2 * (int64_t)mnl + (int64_t)std::max(0, P->m_cap - m_smem) * R;
  P->scratch_stride = (P->scratch_stride + 15) / 16 * 16;
  // ---- checkpoints
  int M = d->ckpt_every;
  if (M == 0) M = std::min(50, P->N);
  if (M < 0) M = 0;
  P->ckpt_every = M;
  P->n_ckpt = M > 0 ? (P->N - 1) / M : 0;
  // ---- device memory
  const int parts = P->n * CL;
  std::vector<double> tabX(P->table.X), tabS(P->table.smax);
  if ((st = upload(P, &P->d_rowptr, rowptr.data(), rowptr.size()))) return st;
  if ((st = upload(P, &P->d_colenc, colenc.data(), colenc.size()))) return st;
  if ((st = upload(P, &P->d_h0v, h0v.data(), h0v.size()))) return st;
  if ((st = upload(P, &P->d_cptr, cptr.data(), cptr.size()))) return st;
  if ((st = upload(P, &P->d_cidx, cidx.data(), cidx.size()))) return st;
  if ((st = upload(P, &P->d_cval, cval.data(), cval.size()))) return st;
  if ((st = upload(P, &P->d_cslice, cslice.data(), cslice.size()))) return st;
  if ((st = upload(P, &P->d_ectr_ptr, ectr_ptr.data(), ectr_ptr.size()))) return st;
  if ((st = upload(P, &P->d_ectr_k, ectr_k.data(), ectr_k.size()))) return st;
  if ((st = upload(P, &P->d_ectr_val, ectr_val.data(), ectr_val.size()))) return st;
  if ((st = upload(P, &P->d_table, tabX.data(), tabX.size()))) return st;
  if ((st = upload(P, &P->d_table_smax, tabS.data(), tabS.size()))) return st;
  const size_t blk = (size_t)dim * P->n;
  if ((st = upload(P, &P->d_psi0, reinterpret_cast<const double2*>(d->psi0), blk))) return st;
  if ((st = upload(P, &P->d_target, reinterpret_cast<const double2*>(d->target), blk))) return st;
  if (d->omega_diag) {
    P->has_omega = true;
    if ((st = upload(P, &P->d_omega, d->omega_diag, (size_t)dim))) return st;
  }
  if ((st = dzeros(P, &P->d_u, (size_t)K * P->N))) return st;
  if ((st = dzeros(P, &P->d_ms_m, (size_t)P->N))) return st;
  if ((st = dzeros(P, &P->d_ms_s, (size_t)P->N))) return st;
  if ((st = dzeros(P, &P->d_norm1, (size_t)P->N))) return st;
  if ((st = dzeros(P, &P->d_psiN, blk))) return st;
  if ((st = dzeros(P, &P->d_ckpt, (size_t)std::max(P->n_ckpt, 1) * blk))) return st;
  if ((st = dzeros(P, &P->d_part_g, (size_t)parts))) return st;
  if ((st = dzeros(P, &P->d_part_c2, (size_t)parts))) return st;
  if ((st = dzeros(P, &P->d_part_grad, (size_t)parts * P->N * std::max(K, 1)))) return st;
  if ((st = dzeros(P, &P->d_g, 1))) return st;
  if ((st = dzeros(P, &P->d_cost, 1))) return st;
  if ((st = dzeros(P, &P->d_parts, 4))) return st;
  if ((st = dzeros(P, &P->d_grad, (size_t)std::max(K, 1) * P->N))) return st;
  if ((st = dzeros(P, &P->d_scratch, (size_t)parts * P->scratch_stride))) return st;
  if ((st = dzeros(P, &P->d_err, 1))) return st;
  return GRAPE_OK;
}

grape::SweepParams sweep_params(grape_problem* P) {
  grape::SweepParams p{};
  p.dim = (int)P->dim;
  p.K = P->K;
  p.N = P->N;
  p.n_states = P->n;
  p.CL = P->CL;
  p.R = P->R;
  p.dt = P->dt;
  p.w_fid = P->w_fid;
  p.w_forbid = P->w_forbid;
  p.w_amp = P->w_amp;
  p.ckpt_every = P->ckpt_every;
  p.n_ckpt = P->n_ckpt;
  p.m_cap = P->m_cap;
  p.rowptr = P->d_rowptr;
  p.colenc = P->d_colenc;
  p.h0v = P->d_h0v;
  p.cptr = P->d_cptr;
  p.cidx = P->d_cidx;
  p.cval = P->d_cval;
  p.cslice = P->d_cslice;
  p.u = P->d_u;
  p.ms_m = P->d_ms_m;
  p.ms_s = P->d_ms_s;
  p.psi0 = P->d_psi0;
  p.target = P->d_target;
  p.omega = P->has_omega ? P->d_omega : nullptr;
  p.psiN = P->d_psiN;
  p.ckpt = P->d_ckpt;
  p.part_g = P->d_part_g;
  p.part_c2 = P->d_part_c2;
  p.part_grad = P->d_part_grad;
  p.g_final = P->d_g;
  p.scratch = P->d_scratch;
  p.scratch_stride = P->scratch_stride;
  p.scr_vals = P->scr_vals;
  p.scr_W = P->scr_W;
  p.scr_wslot = P->scr_wslot;
  p.max_nnz_loc = P->max_nnz_loc;
  p.ectr_ptr = P->d_ectr_ptr;
  p.ectr_k = P->d_ectr_k;
  p.ectr_val = P->d_ectr_val;
  p.err = P->d_err;
  return p;
}

grape_status read_error_word(grape_problem* P, cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  int word = 0;
  e = cudaMemcpy(&word, P->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy (error word)");
  if (word != 0) {
    cudaMemset(P->d_err, 0, sizeof(int));
    switch (word) {
      case grape::kErrTol: return fail(GRAPE_ETOL, "a step has no (m, s) with E_A(m, s) <= tau");
      case grape::kErrNonFinite: return fail(GRAPE_ENONFINITE, "a control amplitude or step norm is not finite");
      case grape::kErrTimeout: return fail(GRAPE_ETIMEOUT, "a bounded device wait gave up");
      default: return fail(GRAPE_ECUDA, "unknown device error word");
    }
  }
  return GRAPE_OK;
}

}  // namespace

extern "C" {

const char* grape_status_string(grape_status st) {
  switch (st) {
    case GRAPE_OK: return "ok";
    case GRAPE_EINVAL: return "invalid argument";
    case GRAPE_ENOMEM: return "out of memory";
    case GRAPE_ECUDA: return "CUDA error";
    case GRAPE_ETOL: return "no (m, s) meets the tolerance";
    case GRAPE_ETIMEOUT: return "device wait timed out";
    case GRAPE_ENOTHERMITIAN: return "operator is not Hermitian";
    case GRAPE_ESTATE: return "call order (grad before cost)";
    case GRAPE_ENONFINITE: return "non-finite control amplitude";
  }
  return "unknown status";
}

const char* grape_last_error(void) { return g_last_error.c_str(); }

int32_t grape_abi_version(void) { return GRAPE_ABI_VERSION; }

double grape_error_bound(double x, int32_t m, int32_t s, int32_t sigma, int32_t precision) {
  return grape::error_bound(x, m, s, sigma, grape::unit_roundoff(precision));
}

grape_status grape_select_ms(double x, double tau, int32_t sigma, int32_t precision, int32_t m_max, int32_t s_max,
                             int32_t* m, int32_t* s) {
  if (!m || !s || !(x >= 0.0) || !(tau > 0.0) || sigma < 1 || m_max < 1 || s_max < 1)
    return fail(GRAPE_EINVAL, "grape_select_ms: bad argument");
  int mm = 0, ss = 0;
  if (!grape::select_ms(x, tau, sigma, grape::unit_roundoff(precision), m_max, s_max, &mm, &ss))
    return fail(GRAPE_ETOL, "no (m, s) pair meets the tolerance");
  *m = mm;
  *s = ss;
  return GRAPE_OK;
}

grape_status grape_problem_create(const grape_desc* d, grape_problem** out) {
  if (!out) return fail(GRAPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(GRAPE_EINVAL, "desc is NULL");
  if (d->dim < 1 || d->dim >= (int64_t)1 << 31) return fail(GRAPE_EINVAL, "dim out of range");
  if (d->n_controls < 0 || d->n_controls > grape::kMaxControls) return fail(GRAPE_EINVAL, "n_controls out of range (0..32)");
  if (d->n_steps < 1) return fail(GRAPE_EINVAL, "n_steps must be >= 1");
  if (d->n_states < 1 || d->n_states > d->dim) return fail(GRAPE_EINVAL, "n_states must be in 1..dim");
  if (!(d->dt > 0.0) || !std::isfinite(d->dt)) return fail(GRAPE_EINVAL, "dt must be finite and > 0");
  if (!(d->tau > 0.0 && d->tau < 1.0)) return fail(GRAPE_EINVAL, "tau must be in (0, 1)");
  if (d->m_max < 0 || d->m_max > grape::kMaxTaylor) return fail(GRAPE_EINVAL, "m_max must be in 0..60");
  if (d->precision != GRAPE_FP64) return fail(GRAPE_EINVAL, "precision: only GRAPE_FP64 is available in this build");
  if (!(d->cluster == 0 || d->cluster == 1 || d->cluster == 2 || d->cluster == 4 || d->cluster == 8 || d->cluster == 16))
    return fail(GRAPE_EINVAL, "cluster must be 0, 1, 2, 4, 8 or 16");
  if (d->n_controls > 0 && !d->Hk) return fail(GRAPE_EINVAL, "Hk is NULL");
  if (!d->psi0 || !d->target) return fail(GRAPE_EINVAL, "psi0 / target is NULL");
  if ((d->alloc == nullptr) != (d->free == nullptr)) return fail(GRAPE_EINVAL, "alloc and free must both be set or both NULL");
  const double ws[3] = {d->w_fid, d->w_forbid, d->w_amp};
  for (double w : ws)
    if (!std::isfinite(w)) return fail(GRAPE_EINVAL, "weights must be finite");
  const size_t blk = (size_t)d->dim * d->n_states * 2;
  for (size_t i = 0; i < blk; ++i)
    if (!std::isfinite(d->psi0[i]) || !std::isfinite(d->target[i])) return fail(GRAPE_EINVAL, "psi0/target not finite");
  if (d->omega_diag)
    for (int64_t i = 0; i < d->dim; ++i)
      if (!std::isfinite(d->omega_diag[i])) return fail(GRAPE_EINVAL, "omega_diag not finite");
  DeviceGuard guard(d->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  grape_problem* P = new (std::nothrow) grape_problem();
  if (!P) return fail(GRAPE_ENOMEM, "host allocation failed");
  P->device = d->device;
  P->dim = d->dim;
  P->K = d->n_controls;
  P->N = d->n_steps;
  P->n = d->n_states;
  P->dt = d->dt;
  P->w_fid = d->w_fid;
  P->w_forbid = d->w_forbid;
  P->w_amp = d->w_amp;
  P->tau = d->tau;
  P->precision = d->precision;
  P->m_cap = d->m_max == 0 ? grape::kMaxTaylor : d->m_max;
  P->alloc_fn = d->alloc;
  P->free_fn = d->free;
  P->alloc_ctx = d->alloc_ctx;
  grape_status st;
  try {
    st = build(P, d);
  } catch (const std::bad_alloc&) {
    st = fail(GRAPE_ENOMEM, "host allocation failed");
  } catch (...) {
    st = fail(GRAPE_EINVAL, "unexpected host error");
  }
  if (st != GRAPE_OK) {
    P->release();
    delete P;
    return st;
  }
  *out = P;
  return GRAPE_OK;
}

void grape_problem_destroy(grape_problem* P) {
  if (!P) return;
  DeviceGuard guard(P->device);
  cudaDeviceSynchronize();
  P->release();
  delete P;
}

}  // extern "C"

namespace {

// Forward sweep (Fig. 1(a)) without host synchronisation; the cost stays on the device.
grape_status run_forward(grape_problem* P, const double* u, bool u_on_device, cudaStream_t st) {
  const size_t ubytes = (size_t)P->K * P->N * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (ubytes)
    e = cudaMemcpyAsync(P->d_u, u, ubytes, u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (u)");
  grape::ScheduleParams sp{};
  sp.dim = (int)P->dim;
  sp.K = P->K;
  sp.N = P->N;
  sp.dt = P->dt;
  sp.rowptr = P->d_rowptr;
  sp.h0v = P->d_h0v;
  sp.ectr_ptr = P->d_ectr_ptr;
  sp.ectr_k = P->d_ectr_k;
  sp.ectr_val = P->d_ectr_val;
  sp.u = P->d_u;
  sp.table = P->d_table;
  sp.table_smax = P->d_table_smax;
  sp.m_cap = P->m_cap;
  sp.s_cap = P->s_cap;
  sp.ms_m = P->d_ms_m;
  sp.ms_s = P->d_ms_s;
  sp.norm1 = P->d_norm1;
  sp.err = P->d_err;
  if ((e = grape::launch_schedule(sp, st)) != cudaSuccess) return cuda_fail(e, "launch k_schedule");
  grape::SweepParams p = sweep_params(P);
  p.in_smem = P->fwd_in_smem;
  p.m_smem = 0;
  if ((e = grape::launch_forward(p, P->precision, P->fwd_smem, P->threads, st)) != cudaSuccess)
    return cuda_fail(e, "launch k_forward");
  grape::FinalizeParams fp{};
  fp.n_parts = P->n * P->CL;
  fp.n_states = P->n;
  fp.N = P->N;
  fp.K = P->K;
  fp.w_fid = P->w_fid;
  fp.w_forbid = P->w_forbid;
  fp.w_amp = P->w_amp;
  fp.part_g = P->d_part_g;
  fp.part_c2 = P->d_part_c2;
  fp.u = P->d_u;
  fp.g_out = P->d_g;
  fp.cost_out = P->d_cost;
  fp.parts_out = P->d_parts;
  if ((e = grape::launch_finalize(fp, st)) != cudaSuccess) return cuda_fail(e, "launch k_finalize");
  P->forward_done = true;
  P->evaluated = true;
  return GRAPE_OK;
}

// Backward sweep (Fig. 1(b)) without host synchronisation; the gradient stays on the device.
grape_status run_backward(grape_problem* P, cudaStream_t st) {
  grape::SweepParams p = sweep_params(P);
  p.in_smem = P->bwd_in_smem;
  p.m_smem = P->m_smem;
  cudaError_t e;
  if ((e = grape::launch_backward(p, P->precision, P->bwd_smem, P->threads, st)) != cudaSuccess)
    return cuda_fail(e, "launch k_backward");
  if (P->K > 0) {
    grape::GradReduceParams gp{};
    gp.n_parts = P->n * P->CL;
    gp.N = P->N;
    gp.K = P->K;
    gp.w_amp = P->w_amp;
    gp.part_grad = P->d_part_grad;
    gp.u = P->d_u;
    gp.grad = P->d_grad;
    if ((e = grape::launch_grad_reduce(gp, st)) != cudaSuccess) return cuda_fail(e, "launch k_grad_reduce");
  }
  return GRAPE_OK;
}

grape_status copy_out(void* dst, const void* src, size_t bytes, bool on_device, cudaStream_t st, const char* what) {
  if (bytes == 0) return GRAPE_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, what);
  return GRAPE_OK;
}

}  // namespace

extern "C" {

grape_status grape_cost(grape_problem* P, const double* u, double* cost, int32_t on_device, void* stream) {
  if (!P || (!u && P->K > 0) || !cost) return fail(GRAPE_EINVAL, "NULL argument");
  DeviceGuard guard(P->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->last_stream = st;
  grape_status s = run_forward(P, u, on_device != 0, st);
  if (s) return s;
  if ((s = copy_out(cost, P->d_cost, sizeof(double), on_device != 0, st, "cudaMemcpyAsync (cost)"))) return s;
  if (!on_device) return read_error_word(P, st);
  return GRAPE_OK;
}

grape_status grape_grad(grape_problem* P, double* grad, int32_t on_device, void* stream) {
  if (!P || (!grad && P->K > 0)) return fail(GRAPE_EINVAL, "NULL argument");
  if (!P->forward_done) return fail(GRAPE_ESTATE, "grape_grad called before grape_cost");
  DeviceGuard guard(P->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->last_stream = st;
  grape_status s = run_backward(P, st);
  if (s) return s;
  if ((s = copy_out(grad, P->d_grad, (size_t)P->K * P->N * sizeof(double), on_device != 0, st, "cudaMemcpyAsync (grad)")))
    return s;
  if (!on_device) return read_error_word(P, st);
  return GRAPE_OK;
}

grape_status grape_cost_and_grad(grape_problem* P, const double* u, double* cost, double* grad, int32_t on_device,
                                 void* stream) {
  if (!P || (!u && P->K > 0) || !cost) return fail(GRAPE_EINVAL, "NULL argument");
  DeviceGuard guard(P->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->last_stream = st;
  grape_status s = run_forward(P, u, on_device != 0, st);
  if (s) return s;
  if (grad) {
    if ((s = run_backward(P, st))) return s;
  }
  if ((s = copy_out(cost, P->d_cost, sizeof(double), on_device != 0, st, "cudaMemcpyAsync (cost)"))) return s;
  if (grad && (s = copy_out(grad, P->d_grad, (size_t)P->K * P->N * sizeof(double), on_device != 0, st,
                            "cudaMemcpyAsync (grad)")))
    return s;
  if (!on_device) return read_error_word(P, st);
  return GRAPE_OK;
}

grape_status grape_sync_status(grape_problem* P, void* stream) {
  if (!P) return fail(GRAPE_EINVAL, "NULL problem");
  DeviceGuard guard(P->device);
  return read_error_word(P, static_cast<cudaStream_t>(stream));
}

grape_status grape_problem_info(grape_problem* P, grape_info* info) {
  if (!P || !info) return fail(GRAPE_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->device_bytes = P->device_bytes;
  info->union_nnz = P->nnz;
  info->ctrl_entries = P->n_ctr;
  info->sigma = P->sigma;
  info->m_cap = P->m_cap;
  info->s_cap = P->s_cap;
  info->cluster = P->CL;
  info->ckpt_every = P->ckpt_every;
  info->smem_bytes = std::max(P->fwd_smem, P->bwd_smem);
  info->total_terms = -1;
  info->max_norm = -1.0;
  if (P->evaluated) {
    DeviceGuard guard(P->device);
    std::vector<int> m(P->N), s(P->N);
    std::vector<double> x(P->N);
    cudaStreamSynchronize(P->last_stream);
    if (cudaMemcpy(m.data(), P->d_ms_m, P->N * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(s.data(), P->d_ms_s, P->N * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(x.data(), P->d_norm1, P->N * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(GRAPE_ECUDA, "cudaMemcpy (schedule)");
    int64_t t = 0;
    double mx = 0.0;
    for (int i = 0; i < P->N; ++i) {
      t += (int64_t)m[i] * s[i];
      mx = std::max(mx, x[i]);
    }
    info->total_terms = t;
    info->max_norm = mx;
  }
  return GRAPE_OK;
}

grape_status grape_step_schedule(grape_problem* P, int32_t* m, int32_t* s, double* norm1) {
  if (!P) return fail(GRAPE_EINVAL, "NULL problem");
  if (!P->evaluated) return fail(GRAPE_ESTATE, "no evaluation has run");
  DeviceGuard guard(P->device);
  cudaError_t e = cudaStreamSynchronize(P->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (m && (e = cudaMemcpy(m, P->d_ms_m, P->N * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (m)");
  if (s && (e = cudaMemcpy(s, P->d_ms_s, P->N * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (s)");
  if (norm1 && (e = cudaMemcpy(norm1, P->d_norm1, P->N * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (norm)");
  return GRAPE_OK;
}

}  // extern "C"
