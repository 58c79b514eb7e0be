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
#include "grape_dense.h"
#include "grape_eig.h"
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

// Partition and shared-memory plan of one sweep kernel.
struct KPlan {
  int CL = 0, R = 0, mnl = 0, threads = 0, smem = 0, in_smem = 0, m_smem = 0;
  int64_t stride = 0, scr_vals = 0, scr_W = 0, scr_Wb = 0, scr_wslot = 0;
  uint32_t* d_colenc = nullptr;
};

struct grape_problem {
  int device = 0;
  int64_t dim = 0;
  int K = 0, N = 0, n = 0;
  double dt = 0, w_fid = 0, w_forbid = 0, w_amp = 0, tau = 0;
  double b_cap = 0;   // cap on ||B||_1 = ||A||_1 / s in the schedule (0 = the paper's rule unchanged)
  double w_tint = 0;  // weight of the time-integrated infidelity C3
  int precision = 0, ckpt_every = 0, n_ckpt = 0, m_cap = 0, s_cap = 0, sigma = 0;
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
  double2* d_h0v = nullptr;
  int* d_cptr = nullptr;
  int* d_cidx = nullptr;
  double2* d_cval = nullptr;
  int* d_cslice = nullptr;   // control slices of the backward partition
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
  double2* d_part_g3 = nullptr;   // per-step overlap partials (C3)
  double2* d_g3 = nullptr;
  double* d_cost = nullptr;
  double* d_parts = nullptr;
  double* d_grad = nullptr;
  double2* d_scratch = nullptr;
  int* d_err = nullptr;
  int bwd_mode = 1;                 // 1 fused (one team per column), 3 three-stage
  // launch plans of the forward and the backward sweep
  KPlan fwd, bwd;
  // three-stage backward (bwd_mode 3): k_costate on the forward's partition, k_gradient on grd;
  // the fused plan bwd stays as the fallback for schedules whose Horner vectors overflow the buffers
  KPlan grd;
  int steps_per_block = 0;
  int64_t hbuf_terms = 0;                // capacity of one block buffer, in terms
  static constexpr int kHbufDepth = 3;   // block buffers of Horner vectors in flight
  static constexpr int kGradStreams = 2; // k_gradient launches alternate between these streams
  void* d_hbuf[kHbufDepth] = {nullptr, nullptr, nullptr};
  double2* d_chi_io = nullptr;           // costate between k_costate launches
  double2* d_seg = nullptr;              // two segments of recomputed states (checkpoints M > 1 apart)
  cudaEvent_t ev_seg[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [slot][gradient stream]
  int* d_plan_flag = nullptr;            // set by k_plan: 1 = the fused fallback runs
  int* d_cslice_g = nullptr;             // control slices of the gradient partition
  cudaStream_t g_stream[kGradStreams] = {nullptr, nullptr};   // k_gradient launches
  cudaEvent_t ev_b = nullptr, ev_g[kHbufDepth] = {nullptr, nullptr, nullptr};
  // A timing event recorded behind every costate launch.  Measured at d = 4000: with it the chain's
  // next launch is not held back behind the gradient kernels (1.96 s per evaluation, against 2.41 s
  // without it or with an event created without timing); nothing reads its timestamp.  Not recorded
  // while a stream is being captured (a recorded graph orders its launches by its own edges).
  cudaEvent_t ev_ct = nullptr;
  int prio_hi = 0;                       // launch priority of the costate chain
  int64_t scr_g_off = 0;                 // k_gradient's regions of d_scratch (double2 units), one of
  int64_t scr_g_size = 0;                // scr_g_size per gradient stream
  // kernel tracing: event pairs around each launch (kind 0..3), summed by grape_kernel_times
  bool tracing = false;
  std::vector<cudaEvent_t> tr_events;    // pool, two per traced launch
  std::vector<int> tr_kind;              // kind of traced launch i (events 2i, 2i+1)
  size_t tr_used = 0;                    // traced launches since the last grape_kernel_times
  // Record the opening event of a traced launch on st; returns its index or -1.
  int trace_begin(int kind, cudaStream_t st) {
    if (!tracing) return -1;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return -1;
    if (2 * (tr_used + 1) > tr_events.size()) {
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t ev = nullptr;
        if (cudaEventCreate(&ev) != cudaSuccess) return -1;
        tr_events.push_back(ev);
      }
      tr_kind.push_back(0);
    }
    const size_t i = tr_used;
    if (cudaEventRecord(tr_events[2 * i], st) != cudaSuccess) return -1;
    tr_kind[i] = kind;
    ++tr_used;
    return (int)i;
  }
  void trace_end(int i, cudaStream_t st) {
    if (i >= 0) cudaEventRecord(tr_events[2 * (size_t)i + 1], st);
  }
  // eigendecomposition propagators (App. F)
  bool eig = false;
  grape::EigCtx ectx{};
  int eig_chunks = 1;                   // step chunks whose propagators are computed concurrently
  std::vector<cudaStream_t> eig_lanes;  // one stream per chunk
  std::vector<cudaEvent_t> eig_ready;   // chunk c's propagators are done
  cudaEvent_t eig_fork = nullptr;
  // dense tensor-core mode
  bool dense = false;
  bool diag_first = false;          // diagonal entries first in their rows (all H_ii real)
  grape::DenseCtx dctx{};
  std::vector<int> m_host, s_host;
  // steepest-descent iteration recorded as a CUDA graph (grape_optimize)
  cudaGraphExec_t opt_exec = nullptr;
  double opt_eta = 0.0;
  double* d_costs = nullptr;
  int d_costs_cap = 0;
  int* d_counter = nullptr;
  // CUDA graphs of the dense sweeps, valid for the schedule they were recorded with
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t fwd_exec = nullptr, bwd_exec = nullptr;
  std::vector<int> fwd_sched, bwd_sched;
  bool forward_done = false;
  bool evaluated = false;
  cudaStream_t last_stream = nullptr;
  int batch_refs = 0;               // batches whose recorded graph refers to this problem's buffers

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
  // Release one allocation made by dalloc (the device must no longer use it).
  void dfree(void* p) {
    for (size_t i = 0; i < allocations.size(); ++i)
      if (allocations[i].first == p) {
        if (free_fn) free_fn(p, allocations[i].second, alloc_ctx);
        else cudaFree(p);
        device_bytes -= (int64_t)allocations[i].second;
        allocations.erase(allocations.begin() + (long)i);
        return;
      }
  }
  void release() {
    for (auto e : tr_events) cudaEventDestroy(e);
    tr_events.clear();
    tr_kind.clear();
    tr_used = 0;
    if (ev_b) cudaEventDestroy(ev_b);
    ev_b = nullptr;
    if (ev_ct) cudaEventDestroy(ev_ct);
    ev_ct = nullptr;
    for (auto& row : ev_seg)
      for (auto& e : row) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
      }
    for (auto& e : ev_g) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    for (auto& g : g_stream) {
      if (g) cudaStreamDestroy(g);
      g = nullptr;
    }
    for (auto e : eig_ready) cudaEventDestroy(e);
    for (auto l : eig_lanes) cudaStreamDestroy(l);
    if (eig_fork) cudaEventDestroy(eig_fork);
    eig_ready.clear();
    eig_lanes.clear();
    eig_fork = nullptr;
    if (opt_exec) cudaGraphExecDestroy(opt_exec);
    opt_exec = nullptr;
    if (fwd_exec) cudaGraphExecDestroy(fwd_exec);
    if (bwd_exec) cudaGraphExecDestroy(bwd_exec);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    fwd_exec = bwd_exec = nullptr;
    cap_stream = nullptr;
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

// Device buffers of the dense tensor-core modes (GRAPE_TC_FP16, GRAPE_TC_BF16).
grape_status build_dense(grape_problem* P, const grape_desc* d, const std::vector<int64_t>& rowptr,
                         const std::vector<int32_t>& ucol, const std::vector<double2>& h0v, const std::vector<int>& cptr,
                         const std::vector<int>& cidx, const std::vector<double2>& cval, const std::vector<int>& ectr_ptr,
                         const std::vector<int>& ectr_k, const std::vector<double2>& ectr_val) {
  grape_status st;
  const int64_t dim = P->dim;
  const int n = P->n, K = P->K, N = P->N;
  P->dense = true;
  P->fwd.CL = P->bwd.CL = 1;   // one partial per reduction
  P->bwd_mode = 1;
  int M = d->ckpt_every;
  if (M == 0) M = std::min(50, N);
  if (M < 0) M = 0;
  P->ckpt_every = M;
  P->n_ckpt = M > 0 ? (N - 1) / M : 0;
  // control-carrying entries and the map from control contributions to them
  std::vector<int> ce_of(rowptr.back(), -1), ce_row, ce_col, cce(cidx.size());
  for (int64_t i = 0; i < dim; ++i)
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e)
      if (ectr_ptr[e + 1] > ectr_ptr[e]) {
        ce_of[e] = (int)ce_row.size();
        ce_row.push_back((int)i);
        ce_col.push_back(ucol[e]);
      }
  for (size_t c = 0; c < cidx.size(); ++c) cce[c] = ce_of[cidx[c]];
  grape::DenseCtx& c = P->dctx;
  c.d = (int)dim;
  c.n = n;
  c.N = N;
  c.K = K;
  c.ksplit = 1;   // chosen below, after the kernel attributes are set
  c.bf16 = P->precision == GRAPE_TC_BF16 ? 1 : 0;
  c.dt = P->dt;
  c.w_fid = P->w_fid;
  c.w_forbid = P->w_forbid;
  c.ckpt_every = P->ckpt_every;
  c.n_ckpt = P->n_ckpt;
  c.inv_fact[0] = 1.0;
  for (int q = 1; q < 62; ++q) c.inv_fact[q] = c.inv_fact[q - 1] / q;
  c.nce = (int)ce_row.size();
  const size_t dd = (size_t)dim * dim, blk = (size_t)dim * n;
  __half* hp[4];
  for (int k = 0; k < 4; ++k)
    if ((st = dzeros(P, &hp[k], dd))) return st;
  c.brh = hp[0];
  c.brl = hp[1];
  c.bih = hp[2];
  c.bil = hp[3];
  __half *xh, *xl;
  // X holds up to 4 n real columns; every TMA box of it (16 rows) and the padded MMA width (a
  // multiple of 16, at most 64) stay inside the allocation
  c.x_rows = std::max(64, (4 * n + 15) / 16 * 16);
  if ((st = dzeros(P, &xh, (size_t)c.x_rows * dim))) return st;
  if ((st = dzeros(P, &xl, (size_t)c.x_rows * dim))) return st;
  c.xh = xh;
  c.xl = xl;
  if ((st = dzeros(P, &xh, (size_t)c.x_rows * dim))) return st;
  if ((st = dzeros(P, &xl, (size_t)c.x_rows * dim))) return st;
  c.xh2 = xh;
  c.xl2 = xl;
  float2* y;
  if ((st = dzeros(P, &y, 2 * blk))) return st;
  c.y = y;
  double2 *psi, *chi, *inc;
  if ((st = dzeros(P, &psi, blk)) || (st = dzeros(P, &chi, blk)) || (st = dzeros(P, &inc, blk))) return st;
  c.psi = psi;
  c.chi = chi;
  c.inc = inc;
  float2 *ws, *xc;
  if ((st = dzeros(P, &ws, (size_t)P->m_cap * blk)) || (st = dzeros(P, &xc, blk))) return st;
  c.wslot = ws;
  c.xcur = xc;
  double2* W;
  if ((st = dzeros(P, &W, (size_t)std::max(c.nce, 1)))) return st;
  c.W = W;
  int *d_cer, *d_cec, *d_cce, *d_ucol;
  if ((st = upload(P, &d_cer, ce_row.data(), std::max<size_t>(ce_row.size(), 1)))) return st;
  if ((st = upload(P, &d_cec, ce_col.data(), std::max<size_t>(ce_col.size(), 1)))) return st;
  if ((st = upload(P, &d_cce, cce.data(), std::max<size_t>(cce.size(), 1)))) return st;
  if ((st = upload(P, &d_ucol, ucol.data(), ucol.size()))) return st;
  c.ce_row = d_cer;
  c.ce_col = d_cec;
  c.cce = d_cce;
  c.ucol = d_ucol;
  std::vector<double> tabX(P->table.X), tabS(P->table.smax);
  if ((st = upload(P, &P->d_rowptr, rowptr.data(), rowptr.size()))) return st;
  if ((st = upload(P, &P->d_h0v, h0v.data(), h0v.size()))) return st;
  if ((st = upload(P, &P->d_cptr, cptr.data(), cptr.size()))) return st;
  if ((st = upload(P, &P->d_cidx, cidx.data(), std::max<size_t>(cidx.size(), 1)))) return st;
  if ((st = upload(P, &P->d_cval, cval.data(), std::max<size_t>(cval.size(), 1)))) return st;
  if ((st = upload(P, &P->d_ectr_ptr, ectr_ptr.data(), ectr_ptr.size()))) return st;
  if ((st = upload(P, &P->d_ectr_k, ectr_k.data(), std::max<size_t>(ectr_k.size(), 1)))) return st;
  if ((st = upload(P, &P->d_ectr_val, ectr_val.data(), std::max<size_t>(ectr_val.size(), 1)))) return st;
  if ((st = upload(P, &P->d_table, tabX.data(), tabX.size()))) return st;
  if ((st = upload(P, &P->d_table_smax, tabS.data(), tabS.size()))) return st;
  if ((st = upload(P, &P->d_psi0, reinterpret_cast<const double2*>(d->psi0), blk))) return st;
  if ((st = upload(P, &P->d_target, reinterpret_cast<const double2*>(d->target), blk))) return st;
  if (d->omega_diag) {
    P->has_omega = true;
    if ((st = upload(P, &P->d_omega, d->omega_diag, (size_t)dim))) return st;
  }
  if ((st = dzeros(P, &P->d_u, (size_t)K * N))) return st;
  if ((st = dzeros(P, &P->d_ms_m, (size_t)N)) || (st = dzeros(P, &P->d_ms_s, (size_t)N)) ||
      (st = dzeros(P, &P->d_norm1, (size_t)N)))
    return st;
  if ((st = dzeros(P, &P->d_psiN, blk)) || (st = dzeros(P, &P->d_ckpt, (size_t)std::max(P->n_ckpt, 1) * blk))) return st;
  if ((st = dzeros(P, &P->d_part_g, 1)) || (st = dzeros(P, &P->d_part_c2, 1))) return st;
  if ((st = dzeros(P, &P->d_part_grad, (size_t)N * std::max(K, 1)))) return st;
  if ((st = dzeros(P, &P->d_g, 1)) || (st = dzeros(P, &P->d_cost, 1)) || (st = dzeros(P, &P->d_parts, 5))) return st;
  if ((st = dzeros(P, &P->d_part_g3, (size_t)N)) || (st = dzeros(P, &P->d_g3, (size_t)N))) return st;
  if ((st = dzeros(P, &P->d_grad, (size_t)std::max(K, 1) * N)) || (st = dzeros(P, &P->d_err, 1))) return st;
  double* c2acc;
  if ((st = dzeros(P, &c2acc, 1))) return st;
  c.c2acc = c2acc;
  c.rowptr = P->d_rowptr;
  c.h0v = P->d_h0v;
  c.ectr_ptr = P->d_ectr_ptr;
  c.ectr_k = P->d_ectr_k;
  c.ectr_val = P->d_ectr_val;
  c.u = P->d_u;
  c.psi0 = P->d_psi0;
  c.target = P->d_target;
  c.omega = P->has_omega ? P->d_omega : nullptr;
  c.psiN = P->d_psiN;
  c.ckpt = P->d_ckpt;
  c.part_g = P->d_part_g;
  c.part_c2 = P->d_part_c2;
  c.g_final = P->d_g;
  c.w_tint = P->w_tint;
  c.part_g3 = P->d_part_g3;
  c.g3 = P->d_g3;
  c.part_grad = P->d_part_grad;
  c.cptr = P->d_cptr;
  c.cval = P->d_cval;
  c.err = P->d_err;
  P->m_host.assign(N, 0);
  P->s_host.assign(N, 0);
  cudaError_t e = grape::dense_prepare();
  if (e != cudaSuccess) return cuda_fail(e, "dense kernel attributes");
  if ((e = grape::dense_make_maps(c)) != cudaSuccess) return cuda_fail(e, "tensor maps of the dense operator");
  c.ksplit = grape::dense_choose_ksplit((int)dim);
  if ((e = cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamCreate");
  return GRAPE_OK;
}

// Device buffers of the eigendecomposition propagator (App. F): dense operators, per-step
// eigenpairs and propagators, the stored state and costate histories.
grape_status build_eig(grape_problem* P, const grape_desc* d, const std::vector<HostCSR>& ops) {
  grape_status st;
  const int64_t dim = P->dim;
  const int n = P->n, K = P->K, N = P->N;
  P->eig = true;
  P->bwd_mode = 1;
  P->ckpt_every = 0;
  P->n_ckpt = 0;
  P->m_cap = P->s_cap = 0;
  const size_t dd = (size_t)dim * dim, blk = (size_t)dim * n;
  std::vector<double2> dense((size_t)(K + 1) * dd, make_double2(0.0, 0.0));
  for (int k = 0; k <= K; ++k)
    for (int64_t i = 0; i < dim; ++i)
      for (int64_t e = ops[k].rowptr[i]; e < ops[k].rowptr[i + 1]; ++e) {
        const cplx v = ops[k].val[e];
        dense[(size_t)k * dd + (size_t)i * dim + ops[k].col[e]] = make_double2(v.real(), v.imag());
      }
  grape::EigCtx& c = P->ectx;
  // CTAs per column in the sweeps: about ten rows each, at most 8 (portable cluster), and no more
  // than the SMs can hold at once for all n columns
  int cl = (int)std::min<int64_t>(8, std::max<int64_t>(1, dim / 10));
  const int nsm = sm_count(P->device);
  while (cl > 1 && (int64_t)n * cl > nsm) --cl;
  c.sweep_cl = cl;
  P->fwd.CL = P->bwd.CL = cl;
  c.d = (int)dim;
  c.n = n;
  c.N = N;
  c.K = K;
  c.dt = P->dt;
  c.w_fid = P->w_fid;
  c.w_forbid = P->w_forbid;
  c.w_tint = P->w_tint;
  // column-wise union pattern of the controls: the entries (a, b) where the gradient needs T_ab
  std::vector<int> cp_ptr(dim + 1, 0), cp_row;
  for (int64_t b = 0; b < dim; ++b) {
    for (int64_t a = 0; a < dim; ++a) {
      bool nz = false;
      for (int k = 1; k <= K && !nz; ++k) {
        const double2 v = dense[(size_t)k * dd + (size_t)a * dim + b];
        nz = v.x != 0.0 || v.y != 0.0;
      }
      if (nz) cp_row.push_back((int)a);
    }
    cp_ptr[b + 1] = (int)cp_row.size();
  }
  int *cp_ptr_d, *cp_row_d;
  if ((st = upload(P, &cp_ptr_d, cp_ptr.data(), cp_ptr.size()))) return st;
  if ((st = upload(P, &cp_row_d, cp_row.data(), std::max<size_t>(cp_row.size(), 1)))) return st;
  c.cp_ptr = cp_ptr_d;
  c.cp_row = cp_row_d;
  double2* ops_d;
  if ((st = upload(P, &ops_d, dense.data(), dense.size()))) return st;
  c.H0 = ops_d;
  c.Hk = ops_d + dd;
  double *lam, *htau;
  double2 *V, *Vt, *U, *ph, *ch, *xs;
  if ((st = dzeros(P, &lam, (size_t)N * dim)) || (st = dzeros(P, &htau, (size_t)N * dim))) return st;
  if ((st = dzeros(P, &V, (size_t)N * dd)) || (st = dzeros(P, &Vt, (size_t)N * dd)) || (st = dzeros(P, &U, (size_t)N * dd)))
    return st;
  if ((st = dzeros(P, &ph, (size_t)(N + 1) * blk)) || (st = dzeros(P, &ch, (size_t)(N + 1) * blk)) ||
      (st = dzeros(P, &xs, (size_t)N * 2 * blk)))
    return st;
  // QR rotations: about d^2 for a whole tridiagonal eigenproblem (1-2 shifted steps per eigenvalue,
  // each one rotation per row of the unreduced block); four times that before the step reports kErrEig
  c.rot_cap = (int)(4 * dd + 64);
  double *tri_a;
  double2 *tri_t, *phase, *rot_cs;
  int *rot_i, *rot_n;
  if ((st = dzeros(P, &tri_a, (size_t)N * dim)) || (st = dzeros(P, &tri_t, (size_t)N * dim)) ||
      (st = dzeros(P, &phase, (size_t)N * dim)) || (st = dzeros(P, &rot_cs, (size_t)N * c.rot_cap)) ||
      (st = dzeros(P, &rot_i, (size_t)N * c.rot_cap)) || (st = dzeros(P, &rot_n, (size_t)N)))
    return st;
  c.tri_a = tri_a;
  c.tri_t = tri_t;
  c.phase = phase;
  c.rot_cs = rot_cs;
  c.rot_i = rot_i;
  c.rot_n = rot_n;
  c.lam = lam;
  c.htau = htau;
  c.V = V;
  c.Vt = Vt;
  c.U = U;
  c.psi_hist = ph;
  c.chi_hist = ch;
  c.xs = xs;
  if ((st = upload(P, &P->d_psi0, reinterpret_cast<const double2*>(d->psi0), blk))) return st;
  if ((st = upload(P, &P->d_target, reinterpret_cast<const double2*>(d->target), blk))) return st;
  if (d->omega_diag) {
    P->has_omega = true;
    if ((st = upload(P, &P->d_omega, d->omega_diag, (size_t)dim))) return st;
  }
  if ((st = dzeros(P, &P->d_u, (size_t)std::max(K, 1) * N))) return st;
  const size_t parts = (size_t)n * cl;
  if ((st = dzeros(P, &P->d_part_g, parts)) || (st = dzeros(P, &P->d_part_c2, parts))) return st;
  if ((st = dzeros(P, &P->d_part_grad, (size_t)N * std::max(K, 1)))) return st;
  if ((st = dzeros(P, &P->d_g, 1)) || (st = dzeros(P, &P->d_cost, 1)) || (st = dzeros(P, &P->d_parts, 5))) return st;
  if ((st = dzeros(P, &P->d_part_g3, parts * N)) || (st = dzeros(P, &P->d_g3, (size_t)N))) return st;
  if ((st = dzeros(P, &P->d_grad, (size_t)std::max(K, 1) * N)) || (st = dzeros(P, &P->d_err, 1))) return st;
  c.psi0 = P->d_psi0;
  c.target = P->d_target;
  c.omega = P->has_omega ? P->d_omega : nullptr;
  c.u = P->d_u;
  c.part_g = P->d_part_g;
  c.part_c2 = P->d_part_c2;
  c.part_g3 = P->w_tint != 0.0 ? P->d_part_g3 : nullptr;
  c.g_final = P->d_g;
  c.g3 = P->d_g3;
  c.part_grad = P->d_part_grad;
  c.err = P->d_err;
  cudaError_t e = grape::eig_prepare((int)dim, K);
  if (e != cudaSuccess) return cuda_fail(e, "eigendecomposition kernel attributes");
  // The QR recurrence of a step is sequential (FP64 latency bound, ~10 ms at d = 80) whatever the
  // number of steps: with the steps in chunks on their own streams, the chunks' reductions,
  // rotations and back-transformations run while other chunks iterate, and the forward sweep
  // starts on a chunk as soon as its propagators are done.
  P->eig_chunks = N >= 256 ? 8 : (N >= 64 ? 4 : 1);
  if (P->eig_chunks > 1) {
    if ((e = cudaEventCreateWithFlags(&P->eig_fork, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    for (int j = 0; j < P->eig_chunks; ++j) {
      cudaStream_t l = nullptr;
      cudaEvent_t ev = nullptr;
      if ((e = cudaStreamCreateWithFlags(&l, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
      P->eig_lanes.push_back(l);
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
      P->eig_ready.push_back(ev);
    }
  }
  return GRAPE_OK;
}

// Eigendecomposition forward pass on st: propagators of every step (in chunks on the problem's
// lanes, forked from and joined back into st) and the forward sweep.
cudaError_t eig_forward_all(grape_problem* P, cudaStream_t st) {
  grape::EigCtx c = P->ectx;
  const int N = P->N, C = P->eig_chunks;
  cudaError_t e;
  if (C <= 1) {
    c.step0 = 0;
    c.nsteps = N;
    if ((e = grape::eig_propagators(c, st)) != cudaSuccess) return e;
    return grape::eig_forward_sweep(c, st);
  }
  if ((e = cudaEventRecord(P->eig_fork, st)) != cudaSuccess) return e;
  for (int j = 0; j < C; ++j) {
    c.step0 = (int)((int64_t)j * N / C);
    c.nsteps = (int)((int64_t)(j + 1) * N / C) - c.step0;
    if ((e = cudaStreamWaitEvent(P->eig_lanes[j], P->eig_fork, 0)) != cudaSuccess) return e;
    if ((e = grape::eig_propagators(c, P->eig_lanes[j])) != cudaSuccess) return e;
    if ((e = cudaEventRecord(P->eig_ready[j], P->eig_lanes[j])) != cudaSuccess) return e;
  }
  for (int j = 0; j < C; ++j) {
    c.step0 = (int)((int64_t)j * N / C);
    c.nsteps = (int)((int64_t)(j + 1) * N / C) - c.step0;
    if ((e = cudaStreamWaitEvent(st, P->eig_ready[j], 0)) != cudaSuccess) return e;
    if ((e = grape::eig_forward_sweep(c, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Record `body` (a sequence of launches on one stream) into a CUDA graph on the problem's capture
// stream, unless `exec` already holds a graph recorded for the same schedule; then launch it on st.
template <typename Body>
cudaError_t run_recorded(grape_problem* P, cudaGraphExec_t* exec, std::vector<int>* sched, cudaStream_t st, Body body) {
  std::vector<int> key(P->m_host);
  key.insert(key.end(), P->s_host.begin(), P->s_host.end());
  cudaError_t e;
  if (!*exec || *sched != key) {
    if (*exec) {
      cudaGraphExecDestroy(*exec);
      *exec = nullptr;
    }
    if ((e = cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t be = body(P->cap_stream);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(P->cap_stream, &g);
    if (be != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return be;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return e;
    *sched = key;
  }
  return cudaGraphLaunch(*exec, st);
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
  if (d->propagator == GRAPE_PROP_EIG) return build_eig(P, d, ops);
  // ---- (m, s) breakpoint table (App. C)
  // Both precisions share the FP64 bound's schedule (the FP32-bulk path keeps its states in FP64;
  // the bound with u = 2^-24 certifies no useful tolerance).
  const double uround = grape::unit_roundoff(GRAPE_FP64);
  P->table = grape::build_table(P->tau, P->sigma, uround, P->m_cap, 4096, 2000.0, P->b_cap > 0.0 ? 128 : 1);
  if (P->table.x_max < 0.0) return fail(GRAPE_ETOL, "no (m, s) pair satisfies E_A <= tau even for ||A||_1 = 0");
  P->m_cap = P->table.m_cap;
  P->s_cap = P->table.s_cap;
  if (P->precision == GRAPE_TC_FP16 || P->precision == GRAPE_TC_BF16)
    return build_dense(P, d, rowptr, ucol, h0v, cptr, cidx, cval, ectr_ptr, ectr_k, ectr_val);
  // ---- row layout.  A Hermitian H_n has a real diagonal: when every operator's stored diagonal is
  // exactly real, B_ii = -i (dt/s) H_ii is imaginary and is stored first in its row.  Off-diagonal
  // entries whose every H_ij term (drift and controls) is real have an imaginary B_ij, those whose
  // every term is imaginary a real B_ij; they follow in two segments, then the general entries.  The
  // one-row-per-thread sweeps apply the first three kinds with two multiplies instead of four; each
  // segment keeps ascending columns, so a CTA's own columns stay contiguous among the general ones.
  bool diag_real = true;
  for (int k = 0; k <= K && diag_real; ++k)
    for (int64_t i = 0; i < dim && diag_real; ++i)
      for (int64_t e = ops[k].rowptr[i]; e < ops[k].rowptr[i + 1]; ++e)
        if (ops[k].col[e] == i && ops[k].val[e].imag() != 0.0) {
          diag_real = false;
          break;
        }
  P->diag_first = diag_real;
  std::vector<uint32_t> eclass(nnz, 0);   // kImagBBit / kRealBBit per entry (new order)
  {
    std::vector<int> seg(nnz, 3);
    for (int64_t e = 0; e < nnz; ++e) {
      bool nonreal = h0v[e].y != 0.0, nonimag = h0v[e].x != 0.0;
      for (auto& pr : per_entry[e]) {
        nonreal = nonreal || pr.second.y != 0.0;
        nonimag = nonimag || pr.second.x != 0.0;
      }
      seg[e] = !nonreal ? 1 : (!nonimag ? 2 : 3);
    }
    std::vector<int64_t> to(nnz), from(nnz);   // new index of an entry, entry at a new index
    std::vector<std::pair<int, int64_t>> key;
    for (int64_t i = 0; i < dim; ++i) {
      const int64_t b = rowptr[i], e = rowptr[i + 1];
      key.clear();
      for (int64_t t = b; t < e; ++t) key.emplace_back(ucol[t] == (int32_t)i && diag_real ? 0 : seg[t], t);
      std::stable_sort(key.begin(), key.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
      for (int64_t t = b; t < e; ++t) {
        from[t] = key[t - b].second;
        to[from[t]] = t;
        const int sg = key[t - b].first;
        eclass[t] = sg == 1 ? grape::kImagBBit : (sg == 2 ? grape::kRealBBit : 0u);
      }
    }
    std::vector<int32_t> ucol2(nnz);
    std::vector<double2> h0v2(nnz);
    for (int64_t t = 0; t < nnz; ++t) {
      ucol2[t] = ucol[from[t]];
      h0v2[t] = h0v[from[t]];
    }
    ucol.swap(ucol2);
    h0v.swap(h0v2);
    for (int k = 0; k < K; ++k) {   // per-control lists: remap, keep them sorted by entry
      std::vector<std::pair<int, double2>> lst;
      for (int c = cptr[k]; c < cptr[k + 1]; ++c) lst.emplace_back((int)to[cidx[c]], cval[c]);
      std::sort(lst.begin(), lst.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
      for (int c = cptr[k]; c < cptr[k + 1]; ++c) {
        cidx[c] = lst[c - cptr[k]].first;
        cval[c] = lst[c - cptr[k]].second;
      }
    }
    ectr_k.clear();
    ectr_val.clear();
    for (int64_t t = 0; t < nnz; ++t) {
      for (auto& pr : per_entry[from[t]]) {
        ectr_k.push_back(pr.first);
        ectr_val.push_back(pr.second);
      }
      ectr_ptr[t + 1] = (int)ectr_k.size();
    }
  }
  // ---- partitions: CTAs per column team (CL) for the forward and the backward sweep.
  // Cost model per Taylor term and CTA, in SM clocks: a * (entries x chains) + b * (rows x chains)
  // + team barrier, with a = 4 FMA per complex multiply-add at 1.7 FP64 lanes/clk (FP32: ~100
  // lanes/clk), b = the FP64 increment of a row, barrier ~80 clk in one CTA and ~1100 clk
  // (barrier + first remote loads) across a cluster; launches wider than the GPU run in waves.
  const int dev = P->device;
  const int nsm = sm_count(dev);
  const int cb = 16;                                          // bytes of one bulk complex number
  const bool stg = P->precision == GRAPE_FP32_BULK;           // compensated FP32 bulk: staged W
  const int smem_max = grape::max_dynamic_smem(dev) - 2048;   // static shared memory of the kernels
  // clocks per complex multiply-add per SM: FP64 4 FMAs (the model's constant from the sweeps' own
  // measured rate); the compensated FP32 one about 48 FP32 operations, whose dependent chains keep
  // the FP32 pipe less than half busy: 105/128 clk, fitted to the three-transmon d = 512 forward
  // (one CTA per column: 2.55 us per term measured against 1.5 us predicted at 48/128; teams of 16,
  // barrier-dominated, matched either way)
  const double a_cost = stg ? 105.0 / 128.0 : 4.0 / 1.7;
  const double b_cost = stg ? 24.0 / 128.0 : 2.0 / 1.7;
  int64_t nnz_ctrl = 0;
  for (int64_t e = 0; e < nnz; ++e) nnz_ctrl += ectr_ptr[e + 1] > ectr_ptr[e] ? 1 : 0;
  const double wf = nnz > 0 ? (double)nnz_ctrl / (double)nnz : 0.0;
  auto rows_entries = [&](int CL, int* R_out, int* mnl_out) -> bool {
    const int64_t R = (dim + CL - 1) / CL;
    if (R >= (1 << 20)) return false;
    int mnl = 0;
    for (int r = 0; r < CL; ++r) {
      const int64_t r0 = std::min<int64_t>((int64_t)r * R, dim), r1 = std::min<int64_t>(r0 + R, dim);
      mnl = std::max<int>(mnl, (int)(rowptr[r1] - rowptr[r0]));
    }
    *R_out = (int)R;
    *mnl_out = std::max(mnl, 1);
    return true;
  };
  auto threads_for = [](int R) { return (int)std::min<int64_t>(512, std::max<int64_t>(64, ((int64_t)R + 31) / 32 * 32)); };
  // fixed cost of one dependent Taylor term (barrier, load and multiply-add latency), measured on GB300
  auto sync_cost = [](int CL) { return CL == 1 ? 1200.0 : 3000.0; };
  auto waves = [&](int ctas) { return std::ceil((double)ctas / nsm); };
  // backward shared-memory plan for (R, mnl): which optional buffers fit, Horner slots kept in smem
  auto bwd_plan = [&](int R, int mnl, int* bin_out, int* msm_out, int* fused_smem, int* split_smem) -> bool {
    if (grape::make_layout(true, R, mnl, 0, 0, cb, stg).total > smem_max) return false;
    int bin = 0;
    if (grape::make_layout(true, R, mnl, 1, 0, cb, stg).total <= smem_max) bin = 1;
    if (grape::make_layout(true, R, mnl, bin | 2, 0, cb, stg).total <= smem_max) bin |= 2;
    if (stg && grape::make_layout(true, R, mnl, bin | 4, 0, cb, stg).total <= smem_max) bin |= 4;
    const int base = grape::make_layout(true, R, mnl, bin, 0, cb, stg).total;
    int msm = (int)std::min<int64_t>(P->m_cap, (smem_max - base - 16) / std::max<int64_t>((int64_t)R * cb, 1));
    msm = std::max(msm, 0);
    *bin_out = bin;
    *msm_out = msm;
    *fused_smem = grape::make_layout(true, R, mnl, bin, msm, cb, stg).total;
    *split_smem = base;
    return true;
  };
  int mode_req = d->backward_mode;

  // forward
  {
    double best = 1e300;
    for (int CL = 1; CL <= grape::kMaxCluster; ++CL) {
      if (d->cluster > 0 && CL != d->cluster) continue;
      if (CL > 1 && CL > dim) continue;
      int R = 0, mnl = 0;
      if (!rows_entries(CL, &R, &mnl)) continue;
      if (grape::make_layout(false, R, mnl, 0, 0, cb, stg).total > smem_max) continue;
      const double cost = waves(P->n * CL) * (a_cost * mnl + b_cost * R + sync_cost(CL));
      // FP64: a larger team must win by 2% (its barriers cost more than the model says); the
      // compensated bulk is latency bound and measured fastest with the largest team that fits
      if (cost < best * (stg ? 1.0 : 0.98)) {
        best = cost;
        P->fwd.CL = CL;
        P->fwd.R = R;
        P->fwd.mnl = mnl;
      }
    }
    if (P->fwd.CL == 0) return fail(GRAPE_EINVAL, "problem does not fit the forward sweep's shared memory");
    const int R = P->fwd.R, mnl = P->fwd.mnl;
    P->fwd.in_smem = grape::make_layout(false, R, mnl, 1, 0, cb, stg).total <= smem_max ? 1 : 0;
    P->fwd.m_smem = 0;
    P->fwd.smem = grape::make_layout(false, R, mnl, P->fwd.in_smem, 0, cb, stg).total;
    P->fwd.threads = threads_for(R);
  }
  // Three-stage backward: the costate chain runs on the forward's partition (n * CL_f SMs), the
  // gradient kernels on whatever is left or after it.  The automatic choice whenever checkpoints are
  // allowed: it measured faster than the fused backward on every workload tried, also where the
  // chain holds most SMs (d = 4000: 2.2x; three transmons, 8 columns x 16 CTAs: 2.0x; d = 16,000,
  // 16 columns x 8 CTAs: 1.3x, the fused backward's 16-CTA teams needing two waves there).
  // Its checkpoint spacing M: every state (M = 1) when they fit 8 GiB, else M = 50, whose segments
  // are recomputed (2 M states held) before the costate chain enters them; an explicit M > 1 asks
  // for that recompute.
  bool three = false;
  int three_M = 1;
  {
    const double state_bytes = (double)P->N * (double)dim * P->n * 16.0;
    if (mode_req == 3) three = true;
    else if (mode_req == 0)
      three = d->ckpt_every >= 0 && P->N >= 2;
    if (three) three_M = d->ckpt_every > 0 ? d->ckpt_every : (state_bytes <= 8.0 * (1 << 30) ? 1 : 50);
    three_M = std::max(1, std::min(three_M, P->N));
  }
  // k_gradient partition: the smallest team that fits shared memory at all (its exchange buffers,
  // states and pattern; values and W accumulators join them when they fit, else they stay in the
  // CTA's global scratch slice, which the L2 holds).  The gradient kernel is throughput bound: the
  // fewer CTAs per team, the fewer barriers and remote loads per unit of work (measured at
  // d = 4000: teams of 2 CTAs beat 4, 8 and 16).  Blocks of steps are long enough that a block's
  // gradient work covers about twice the SMs the costate chain leaves free.
  if (three) {
    int pick = 0, pick_in = 0;
    const int full = 1 | 2 | (stg ? 4 : 0);
    // The compensated bulk's accumulations are cheap enough that W and value traffic to global
    // scratch would dominate: it first looks for the smallest team that holds everything.
    for (int pass = stg ? 0 : 1; pass < 2 && !pick; ++pass)
      for (int CL = 1; CL <= grape::kMaxCluster && !pick; ++CL) {
        if (d->grad_cluster > 0 && CL != d->grad_cluster) continue;
        if (CL > 1 && CL > dim) continue;
        int R = 0, mnl = 0;
        if (!rows_entries(CL, &R, &mnl)) continue;
        for (int want : {full, 2 | (stg ? 4 : 0), 0}) {
          if (pass == 0 && want != full) break;
          if (grape::make_glayout(R, mnl, want, cb, stg).total > smem_max) continue;
          pick = CL;
          pick_in = want;
          P->grd.R = R;
          P->grd.mnl = mnl;
          break;
        }
      }
    if (!pick) {
      if (mode_req == 3) return fail(GRAPE_EINVAL, "backward_mode 3: the gradient kernel does not fit shared memory");
      three = false;
    } else {
      P->grd.CL = pick;
      P->grd.in_smem = pick_in;
      P->grd.m_smem = 0;
      P->grd.smem = grape::make_glayout(P->grd.R, P->grd.mnl, pick_in, cb, stg).total;
      P->grd.threads = threads_for(P->grd.R);
      const int free_sms = std::max(nsm - P->n * P->fwd.CL, P->n * pick);
      int S = d->block_steps > 0 ? d->block_steps : std::min(32, std::max(1, 2 * free_sms / (P->n * pick)));
      S = std::min(S, P->N);
      // with recomputed segments, blocks must not straddle them: the largest divisor of M not above S
      if (three_M > 1) {
        S = std::min(S, three_M);
        while (three_M % S) --S;
      }
      P->steps_per_block = S;
    }
  }
  // backward: one team per column (fused); with the three-stage backward, the fused plan is its fallback
  if (three) mode_req = 1;
  {
    double best = 1e300;
    for (int CL = 1; CL <= grape::kMaxCluster; ++CL) {
      if (d->cluster > 0 && CL != d->cluster) continue;
      if (CL > 1 && CL > dim) continue;
      int R = 0, mnl = 0, bin = 0, msm = 0, fsm = 0, ssm = 0;
      if (!rows_entries(CL, &R, &mnl)) continue;
      if (!bwd_plan(R, mnl, &bin, &msm, &fsm, &ssm)) continue;
      const int thr = threads_for(R);
      (void)ssm;
      const double cost = waves(P->n * CL) * (a_cost * mnl * (3.0 + wf) + b_cost * R * 2.0 + 2.0 * sync_cost(CL));
      if (cost < best * 0.98) {
        best = cost;
        P->bwd_mode = 1;
        P->bwd.CL = CL;
        P->bwd.R = R;
        P->bwd.mnl = mnl;
        P->bwd.in_smem = bin;
        P->bwd.m_smem = msm;
        P->bwd.smem = fsm;
        P->bwd.threads = thr;
      }
    }
    if (P->bwd.CL == 0) return fail(GRAPE_EINVAL, "problem does not fit the backward sweep's shared memory");
  }
  if (three) P->bwd_mode = 3;
  // column encodings (owner CTA, local row, control bit) of both partitions, control slices of the backward one
  auto encode = [&](int R, std::vector<uint32_t>& enc) {
    enc.resize(nnz);
    for (int64_t i = 0; i < dim; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t j = ucol[e];
        const uint32_t owner = (uint32_t)(j / R), local = (uint32_t)(j - (int64_t)owner * R);
        uint32_t x = (owner << grape::kOwnerShift) | local | eclass[e];
        if (ectr_ptr[e + 1] > ectr_ptr[e]) x |= grape::kCtrlBit;
        enc[e] = x;
      }
  };
  std::vector<uint32_t> colenc_f, colenc_b, colenc_g;
  encode(P->fwd.R, colenc_f);
  encode(P->bwd.R, colenc_b);
  if (three) encode(P->grd.R, colenc_g);
  auto slices = [&](int CLx, int Rx, std::vector<int>& cs) {
    cs.assign((size_t)std::max(K, 1) * CLx * 2, 0);
    for (int k = 0; k < K; ++k)
      for (int r = 0; r < CLx; ++r) {
        const int64_t r0 = std::min<int64_t>((int64_t)r * Rx, dim), r1 = std::min<int64_t>(r0 + Rx, dim);
        const auto b = cidx.begin() + cptr[k], e = cidx.begin() + cptr[k + 1];
        cs[(k * CLx + r) * 2] = (int)(std::lower_bound(b, e, (int)rowptr[r0]) - cidx.begin());
        cs[(k * CLx + r) * 2 + 1] = (int)(std::lower_bound(b, e, (int)rowptr[r1]) - cidx.begin());
      }
  };
  std::vector<int> cslice, cslice_g;
  slices(P->bwd.CL, P->bwd.R, cslice);
  if (three) slices(P->grd.CL, P->grd.R, cslice_g);
  // per-CTA global scratch (buffers that do not fit in shared memory), in double2 units
  for (KPlan* kp : {&P->fwd, &P->bwd, &P->grd}) {
    if (kp->CL == 0) continue;
    kp->scr_vals = 0;
    kp->scr_W = kp->mnl;
    kp->scr_Wb = 2 * (int64_t)kp->mnl;
    kp->scr_wslot = 3 * (int64_t)kp->mnl;
    const int wslots = kp == &P->bwd ? std::max(0, P->m_cap - kp->m_smem) : 0;
    kp->stride = (3 * (int64_t)kp->mnl + (int64_t)wslots * kp->R + 15) / 16 * 16;
  }
  // ---- checkpoints
  int M = d->ckpt_every;
  if (M == 0) M = three ? three_M : std::min(50, P->N);
  if (three) M = three_M;
  if (M < 0) M = 0;
  P->ckpt_every = M;
  P->n_ckpt = M > 0 ? (P->N - 1) / M : 0;
  // ---- device memory
  const int parts_f = P->n * P->fwd.CL, parts_b = std::max(P->n * P->bwd.CL, P->n * P->grd.CL);
  std::vector<double> tabX(P->table.X), tabS(P->table.smax);
  if ((st = upload(P, &P->d_rowptr, rowptr.data(), rowptr.size()))) return st;
  if ((st = upload(P, &P->fwd.d_colenc, colenc_f.data(), colenc_f.size()))) return st;
  if ((st = upload(P, &P->bwd.d_colenc, colenc_b.data(), colenc_b.size()))) return st;
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
  if ((st = dzeros(P, &P->d_part_g, (size_t)parts_f))) return st;
  if ((st = dzeros(P, &P->d_part_c2, (size_t)parts_f))) return st;
  if ((st = dzeros(P, &P->d_part_grad, (size_t)parts_b * P->N * std::max(K, 1)))) return st;
  if ((st = dzeros(P, &P->d_g, 1))) return st;
  if ((st = dzeros(P, &P->d_cost, 1))) return st;
  if ((st = dzeros(P, &P->d_parts, 5))) return st;
  if ((st = dzeros(P, &P->d_grad, (size_t)std::max(K, 1) * P->N))) return st;
  if ((st = dzeros(P, &P->d_err, 1))) return st;
  if ((st = dzeros(P, &P->d_part_g3, (size_t)parts_f * P->N)) || (st = dzeros(P, &P->d_g3, (size_t)P->N))) return st;
  const int64_t scr_f = (int64_t)parts_f * P->fwd.stride;
  const int64_t scr_b = (int64_t)P->n * P->bwd.CL * P->bwd.stride;
  // k_costate (forward partition) and the k_gradient launches of the gradient streams run at the
  // same time: disjoint scratch regions, one per gradient stream
  int64_t scr_g = 0;
  if (three) scr_g = (int64_t)P->steps_per_block * P->n * P->grd.CL * P->grd.stride;
  P->scr_g_off = scr_f;
  P->scr_g_size = scr_g;
  const int64_t scr_three = scr_f + grape_problem::kGradStreams * scr_g;
  if ((st = dzeros(P, &P->d_scratch, (size_t)std::max(scr_three, scr_b)))) return st;
  if (three) {
    // Block buffers of Horner vectors, first sized for the schedule of 1.25 times the drift's norm (at
    // least 2 m_cap terms per step).  Outside stream capture every evaluation reads its schedule back
    // and grows them when a block needs more; under capture k_plan selects the fused fallback for a
    // schedule that does not fit.
    double xd = 0.0;
    for (int64_t i = 0; i < dim; ++i) {
      double a = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) a += std::hypot(h0v[e].x, h0v[e].y);
      xd = std::max(xd, a);
    }
    auto mu_of = [&](double x) -> int64_t {
      int s0 = 1;
      if (P->b_cap > 0.0) s0 = std::max(1, (int)std::ceil(x / P->b_cap));
      for (int s1 = s0; s1 <= P->s_cap; ++s1)
        if (P->table.smax[s1 - 1] >= x)
          for (int m1 = 1; m1 <= P->m_cap; ++m1)
            if (P->table.X[(size_t)(s1 - 1) * P->m_cap + (m1 - 1)] >= x) return (int64_t)m1 * s1;
      return 0;
    };
    const int64_t mu = std::max<int64_t>(mu_of(1.25 * P->dt * xd), 2 * P->m_cap);
    P->hbuf_terms = mu * P->steps_per_block;
    P->m_host.assign(P->N, 0);
    P->s_host.assign(P->N, 0);
    const size_t hb = (size_t)P->hbuf_terms * (size_t)dim * P->n * (size_t)cb;
    for (auto& h : P->d_hbuf) {
      h = P->dalloc(hb);
      if (!h) return fail(GRAPE_ENOMEM, "device allocation failed");
    }
    if ((st = upload(P, &P->grd.d_colenc, colenc_g.data(), colenc_g.size()))) return st;
    if ((st = upload(P, &P->d_cslice_g, cslice_g.data(), cslice_g.size()))) return st;
    if ((st = dzeros(P, &P->d_chi_io, blk))) return st;
    if ((st = dzeros(P, &P->d_plan_flag, 1))) return st;
    if (M > 1 && (st = dzeros(P, &P->d_seg, (size_t)2 * M * blk))) return st;
    int lo = 0, hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetStreamPriorityRange");
    P->prio_hi = hi;
    for (auto& g : P->g_stream)
      if ((e = cudaStreamCreateWithPriority(&g, cudaStreamNonBlocking, lo)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreateWithPriority");
    if ((e = cudaEventCreateWithFlags(&P->ev_b, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreateWithFlags");
    if ((e = cudaEventCreate(&P->ev_ct)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    for (auto& ev : P->ev_g)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreateWithFlags");
    for (auto& row : P->ev_seg)
      for (auto& ev : row)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
          return cuda_fail(e, "cudaEventCreateWithFlags");
  }
  return GRAPE_OK;
}

grape::SweepParams sweep_params(grape_problem* P, const KPlan& kp) {
  grape::SweepParams p{};
  p.dim = (int)P->dim;
  p.K = P->K;
  p.N = P->N;
  p.n_states = P->n;
  p.CL = kp.CL;
  p.R = kp.R;
  p.dt = P->dt;
  p.w_fid = P->w_fid;
  p.w_forbid = P->w_forbid;
  p.w_amp = P->w_amp;
  p.w_tint = P->w_tint;
  p.part_g3 = P->d_part_g3;
  p.g3 = P->d_g3;
  p.ckpt_every = P->ckpt_every;
  p.n_ckpt = P->n_ckpt;
  p.m_cap = P->m_cap;
  p.diag_first = P->diag_first ? 1 : 0;
  p.rowptr = P->d_rowptr;
  p.colenc = kp.d_colenc;
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
  p.scratch_stride = kp.stride;
  p.scr_vals = kp.scr_vals;
  p.scr_W = kp.scr_W;
  p.scr_Wb = kp.scr_Wb;
  p.scr_wslot = kp.scr_wslot;
  p.max_nnz_loc = kp.mnl;
  p.in_smem = kp.in_smem;
  p.m_smem = kp.m_smem;
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
      case grape::kErrEig: return fail(GRAPE_ETOL, "the tridiagonal QR iteration of a step did not converge");
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
  if (d->precision != GRAPE_FP64 && d->precision != GRAPE_FP32_BULK && d->precision != GRAPE_TC_FP16 &&
      d->precision != GRAPE_TC_BF16)
    return fail(GRAPE_EINVAL, "precision must be GRAPE_FP64, GRAPE_FP32_BULK, GRAPE_TC_FP16 or GRAPE_TC_BF16");
  if ((d->precision == GRAPE_TC_FP16 || d->precision == GRAPE_TC_BF16) && (d->dim % 128 != 0 || d->n_states > 16))
    return fail(GRAPE_EINVAL, "the tensor-core modes need dim % 128 == 0 and n_states <= 16");
  if (d->propagator != GRAPE_PROP_TAYLOR && d->propagator != GRAPE_PROP_EIG)
    return fail(GRAPE_EINVAL, "propagator must be GRAPE_PROP_TAYLOR or GRAPE_PROP_EIG");
  if (d->propagator == GRAPE_PROP_EIG && (d->precision != GRAPE_FP64 || d->dim > grape::kEigMaxDim))
    return fail(GRAPE_EINVAL, "GRAPE_PROP_EIG needs GRAPE_FP64 and dim <= 96");
  if (d->cluster < 0 || d->cluster > grape::kMaxCluster) return fail(GRAPE_EINVAL, "cluster must be 0 (automatic) or 1..16");
  if (d->backward_mode < 0 || d->backward_mode > 3 || d->backward_mode == 2)
    return fail(GRAPE_EINVAL, "backward_mode must be 0 (automatic), 1 (one team per column) or 3 (three-stage)");
  if (d->backward_mode == 3 && d->ckpt_every < 0)
    return fail(GRAPE_EINVAL, "backward_mode 3 needs checkpoints: ckpt_every must be >= 0");
  if (d->grad_cluster < 0 || d->grad_cluster > grape::kMaxCluster)
    return fail(GRAPE_EINVAL, "grad_cluster must be 0 (automatic) or 1..16");
  if (d->block_steps < 0) return fail(GRAPE_EINVAL, "block_steps must be >= 0");
  if (d->n_controls > 0 && !d->Hk) return fail(GRAPE_EINVAL, "Hk is NULL");
  if (d->bulk_norm_cap < 0.0 || !std::isfinite(d->bulk_norm_cap)) return fail(GRAPE_EINVAL, "bulk_norm_cap must be >= 0");
  if (!d->psi0 || !d->target) return fail(GRAPE_EINVAL, "psi0 / target is NULL");
  if ((d->alloc == nullptr) != (d->free == nullptr)) return fail(GRAPE_EINVAL, "alloc and free must both be set or both NULL");
  const double ws[4] = {d->w_fid, d->w_forbid, d->w_amp, d->w_tint};
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
  P->w_tint = d->w_tint;
  P->tau = d->tau;
  P->precision = d->precision;
  P->m_cap = d->m_max == 0 ? grape::kMaxTaylor : d->m_max;
  const bool tc = d->precision == GRAPE_TC_FP16 || d->precision == GRAPE_TC_BF16;
  P->b_cap = d->bulk_norm_cap > 0.0 ? d->bulk_norm_cap : (tc ? 2.0 : 0.0);
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

grape::ScheduleParams schedule_params(const grape_problem* P) {
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
  sp.b_cap = P->b_cap;
  return sp;
}

// The cost from the forward sweep's n_parts partials (Sec. II composite cost).
grape::FinalizeParams finalize_params(const grape_problem* P, int n_parts) {
  grape::FinalizeParams fp{};
  fp.n_parts = n_parts;
  fp.n_states = P->n;
  fp.N = P->N;
  fp.K = P->K;
  fp.w_fid = P->w_fid;
  fp.w_forbid = P->w_forbid;
  fp.w_amp = P->w_amp;
  fp.w_tint = P->w_tint;
  fp.part_g3 = P->w_tint != 0.0 ? P->d_part_g3 : nullptr;
  fp.g3_out = P->d_g3;
  fp.part_g = P->d_part_g;
  fp.part_c2 = P->d_part_c2;
  fp.u = P->d_u;
  fp.g_out = P->d_g;
  fp.cost_out = P->d_cost;
  fp.parts_out = P->d_parts;
  return fp;
}

// dC/du_kn from the backward sweep's n_parts partials plus the amplitude term 2 w_amp u_kn / N (App. A).
grape::GradReduceParams grad_reduce_params(const grape_problem* P, int n_parts) {
  grape::GradReduceParams gp{};
  gp.n_parts = n_parts;
  gp.N = P->N;
  gp.K = P->K;
  gp.w_amp = P->w_amp;
  gp.part_grad = P->d_part_grad;
  gp.u = P->d_u;
  gp.grad = P->d_grad;
  return gp;
}

// Forward sweep (Fig. 1(a)) without host synchronisation; the cost stays on the device.
grape_status run_forward(grape_problem* P, const double* u, bool u_on_device, cudaStream_t st) {
  const size_t ubytes = (size_t)P->K * P->N * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (ubytes && u != P->d_u)
    e = cudaMemcpyAsync(P->d_u, u, ubytes, u_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (u)");
  if (P->eig) {
    if ((e = grape::check_nonfinite_u(P->d_u, (int64_t)P->K * P->N, P->d_err, st)) != cudaSuccess)
      return cuda_fail(e, "launch k_check_finite");
    if ((e = eig_forward_all(P, st)) != cudaSuccess) return cuda_fail(e, "eigendecomposition forward sweep");
    const grape::FinalizeParams fp = finalize_params(P, P->n * P->ectx.sweep_cl);
    if ((e = grape::launch_finalize(fp, st)) != cudaSuccess) return cuda_fail(e, "launch k_finalize");
    P->forward_done = true;
    P->evaluated = true;
    return GRAPE_OK;
  }
  const grape::ScheduleParams sp = schedule_params(P);
  if ((e = grape::launch_schedule(sp, st)) != cudaSuccess) return cuda_fail(e, "launch k_schedule");
  if (P->dense) {
    // the host drives one tensor-core product per Taylor term: it needs the schedule
    if ((e = cudaMemcpyAsync(P->m_host.data(), P->d_ms_m, P->N * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(P->s_host.data(), P->d_ms_s, P->N * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return cuda_fail(e, "schedule download");
    e = run_recorded(P, &P->fwd_exec, &P->fwd_sched, st, [&](cudaStream_t cs) {
      return grape::dense_forward(P->dctx, P->m_host.data(), P->s_host.data(), cs);
    });
    if (e != cudaSuccess) return cuda_fail(e, "dense forward sweep");
    const grape::FinalizeParams fp = finalize_params(P, 1);
    if ((e = grape::launch_finalize(fp, st)) != cudaSuccess) return cuda_fail(e, "launch k_finalize");
    P->forward_done = true;
    P->evaluated = true;
    return GRAPE_OK;
  }
  grape::SweepParams p = sweep_params(P, P->fwd);
  const int tf = P->trace_begin(0, st);
  if ((e = grape::launch_forward(p, P->precision, P->fwd.smem, P->fwd.threads, st)) != cudaSuccess)
    return cuda_fail(e, "launch k_forward");
  P->trace_end(tf, st);
  const grape::FinalizeParams fp = finalize_params(P, P->n * P->fwd.CL);
  if ((e = grape::launch_finalize(fp, st)) != cudaSuccess) return cuda_fail(e, "launch k_finalize");
  P->forward_done = true;
  P->evaluated = true;
  return GRAPE_OK;
}

// Backward sweep (Fig. 1(b)) without host synchronisation; the gradient stays on the device.
grape_status run_backward(grape_problem* P, cudaStream_t st) {
  grape::SweepParams p = sweep_params(P, P->bwd);
  cudaError_t e;
  if (P->eig) {
    if ((e = grape::eig_backward(P->ectx, st)) != cudaSuccess) return cuda_fail(e, "eigendecomposition backward sweep");
  } else if (P->dense) {
    e = run_recorded(P, &P->bwd_exec, &P->bwd_sched, st, [&](cudaStream_t cs) {
      return grape::dense_backward(P->dctx, P->m_host.data(), P->s_host.data(), cs);
    });
    if (e != cudaSuccess) return cuda_fail(e, "dense backward sweep");
  } else if (P->bwd_mode == 3) {
    // k_plan decides whether the block buffers hold this schedule's Horner vectors.  Then, per block
    // of steps (descending), the costate chain on the caller's stream (high launch priority) and the
    // gradient kernel of the block on one of the gradient streams (alternating, so that consecutive
    // blocks' gradient kernels overlap and fill the SMs the chain leaves) once the chain has stored
    // the block; kHbufDepth buffers rotate, so the chain waits for the gradient kernel of the block
    // kHbufDepth ahead.  The fused backward is queued after the join and returns at once unless
    // k_plan selected it.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap == cudaStreamCaptureStatusNone) {
      // the schedule of this evaluation (k_schedule ran before the forward sweep)
      if ((e = cudaMemcpyAsync(P->m_host.data(), P->d_ms_m, P->N * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(P->s_host.data(), P->d_ms_s, P->N * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "schedule download");
      int64_t need = 0;
      for (int b0 = 0; b0 < P->N; b0 += P->steps_per_block) {
        int64_t t = 0;
        for (int n = b0; n < std::min(P->N, b0 + P->steps_per_block); ++n)
          if (P->m_host[n] > 0 && P->s_host[n] > 0) t += (int64_t)P->m_host[n] * P->s_host[n];
        need = std::max(need, t);
      }
      // A recorded batch refers to the current buffers: they are not replaced while one exists (k_plan
      // then selects the fused backward for a schedule that does not fit).
      if (need > P->hbuf_terms && P->batch_refs == 0) {   // the stream was just synchronised
        if (P->opt_exec) {            // a recorded optimizer iteration refers to the old buffers
          cudaGraphExecDestroy(P->opt_exec);
          P->opt_exec = nullptr;
        }
        const int64_t terms = need + need / 4;
        const size_t cbytes = 16;   // one bulk complex (double2, or float4 for the compensated bulk)
        const size_t hb = (size_t)terms * (size_t)P->dim * P->n * cbytes;
        for (auto& h : P->d_hbuf) {
          P->dfree(h);
          h = P->dalloc(hb);
          if (!h) {
            for (auto& h2 : P->d_hbuf) { P->dfree(h2); h2 = nullptr; }
            P->bwd_mode = 1;   // no room for the block buffers: the fused backward from now on
            break;
          }
        }
        if (P->bwd_mode == 3) P->hbuf_terms = terms;
      }
    }
    if (P->bwd_mode != 3) return run_backward(P, st);
    grape::PlanParams pp{};
    pp.N = P->N;
    pp.steps_per_block = P->steps_per_block;
    pp.cap_terms = P->hbuf_terms;
    pp.ms_m = P->d_ms_m;
    pp.ms_s = P->d_ms_s;
    pp.flag = P->d_plan_flag;
    if ((e = grape::launch_plan(pp, st)) != cudaSuccess) return cuda_fail(e, "launch k_plan");
    grape::SweepParams pc = sweep_params(P, P->fwd);
    pc.chi_io = P->d_chi_io;
    pc.plan_flag = P->d_plan_flag;
    pc.hbuf_terms = P->hbuf_terms;
    grape::SweepParams pg = sweep_params(P, P->grd);
    pg.cslice = P->d_cslice_g;
    double2* const scr_g0 = P->d_scratch + P->scr_g_off;
    pg.plan_flag = P->d_plan_flag;
    pg.hbuf_terms = P->hbuf_terms;
    const int S = P->steps_per_block, nb = (P->N + S - 1) / S;
    constexpr int D = grape_problem::kHbufDepth, G = grape_problem::kGradStreams;
    // Checkpoints M > 1 apart: before the costate chain enters segment j = [j M, (j+1) M), a
    // forward launch recomputes the segment's states from its checkpoint into slot j % 2 of the
    // segment buffer, once the gradient kernels of segment j + 2 (the slot's previous user) are done.
    const int Mseg = P->ckpt_every;
    const bool segs = Mseg > 1;
    const int last_seg = segs ? (P->N - 1) / Mseg : 0;
    if (segs) {
      pc.seg = pg.seg = P->d_seg;
      pc.seg_M = pg.seg_M = Mseg;
    }
    int cur_seg = -1;
    for (int b = nb - 1; b >= 0; --b) {
      const int slot = b % D;
      cudaStream_t gs = P->g_stream[b % G];
      const int jseg = segs ? (b * S) / Mseg : 0;
      if (segs && jseg != cur_seg) {
        if (jseg + 2 <= last_seg)
          for (int g = 0; g < G; ++g)
            if ((e = cudaStreamWaitEvent(st, P->ev_seg[jseg & 1][g], 0)) != cudaSuccess)
              return cuda_fail(e, "cudaStreamWaitEvent");
        grape::SweepParams pr = sweep_params(P, P->fwd);
        pr.recompute = 1;
        pr.seg = P->d_seg;
        pr.seg_M = Mseg;
        pr.n_begin = jseg * Mseg;
        pr.n_end = std::min((jseg + 1) * Mseg, P->N) - 1;
        pr.rec_src = jseg == 0 ? P->d_psi0 : P->d_ckpt + (size_t)(jseg - 1) * P->n * P->dim;
        const int tr = P->trace_begin(4, st);
        if ((e = grape::launch_forward(pr, P->precision, P->fwd.smem, P->fwd.threads, st)) != cudaSuccess)
          return cuda_fail(e, "launch k_forward (segment recompute)");
        P->trace_end(tr, st);
        cur_seg = jseg;
      }
      pg.scratch = scr_g0 + (int64_t)(b % G) * P->scr_g_size;   // concurrent launches never share scratch
      pc.n_begin = pg.n_begin = b * S;
      pc.n_end = pg.n_end = std::min(P->N, (b + 1) * S);
      pc.hbuf = pg.hbuf = P->d_hbuf[slot];
      if (b + D <= nb - 1 && (e = cudaStreamWaitEvent(st, P->ev_g[slot], 0)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamWaitEvent");
      const int tc = P->trace_begin(1, st);
      if ((e = grape::launch_costate(pc, P->precision, P->fwd.smem, P->fwd.threads, P->prio_hi, st)) != cudaSuccess)
        return cuda_fail(e, "launch k_costate");
      P->trace_end(tc, st);
      if (cap == cudaStreamCaptureStatusNone && (e = cudaEventRecord(P->ev_ct, st)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord");
      if ((e = cudaEventRecord(P->ev_b, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
      if ((e = cudaStreamWaitEvent(gs, P->ev_b, 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
      const int tg = P->trace_begin(2, gs);
      if ((e = grape::launch_gradient(pg, P->precision, P->grd.smem, P->grd.threads, gs)) != cudaSuccess)
        return cuda_fail(e, "launch k_gradient");
      P->trace_end(tg, gs);
      if ((e = cudaEventRecord(P->ev_g[slot], gs)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
      if (segs && b * S == jseg * Mseg)   // the segment's last block: mark its gradient work on each stream
        for (int g = 0; g < G; ++g)
          if ((e = cudaEventRecord(P->ev_seg[jseg & 1][g], P->g_stream[g])) != cudaSuccess)
            return cuda_fail(e, "cudaEventRecord");
    }
    // join: the last gradient kernel of each stream (blocks 0 .. G-1, slots b % D)
    for (int b = 0; b < std::min(G, nb); ++b)
      if ((e = cudaStreamWaitEvent(st, P->ev_g[b % D], 0)) != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
    grape::SweepParams pf = sweep_params(P, P->bwd);
    pf.plan_flag = P->d_plan_flag;
    pf.gate_on_flag = 1;
    if ((e = grape::launch_backward(pf, P->precision, P->bwd.smem, P->bwd.threads, st)) != cudaSuccess)
      return cuda_fail(e, "launch k_backward (fallback)");
  } else {
    const int tb = P->trace_begin(3, st);
    if ((e = grape::launch_backward(p, P->precision, P->bwd.smem, P->bwd.threads, st)) != cudaSuccess)
      return cuda_fail(e, "launch k_backward");
    P->trace_end(tb, st);
  }
  if (P->K > 0) {
    grape::GradReduceParams gp = grad_reduce_params(P, (P->dense || P->eig) ? 1 : P->n * P->bwd.CL);
    if (!P->dense && !P->eig && P->bwd_mode == 3) {
      gp.n_parts = P->n * P->grd.CL;
      gp.n_parts_alt = P->n * P->bwd.CL;
      gp.plan_flag = P->d_plan_flag;
    }
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

// ------------------------------------------------------------------ batches

}  // extern "C"

struct grape_batch {
  int device = 0;
  int count = 0;
  std::vector<grape_problem*> probs;
  std::vector<int64_t> u_off, g_off;
  int64_t u_total = 0, g_total = 0;
  double* d_u = nullptr;
  double* d_cost = nullptr;
  double* d_grad = nullptr;
  std::vector<void*> owned;                 // cudaMalloc'ed staging and queue buffers
  cudaStream_t origin = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int> order;                   // lane members, longest first
  std::vector<int> lane;                    // stream of each lane member
  std::vector<char> queued;                 // member runs in the work queue
  // Work queue, one per bulk precision among the queued members: k_schedule_batch, then one
  // persistent k_queue launch per sweep direction over (member, column) items, longest first.
  struct Queue {
    int precision = 0;
    std::vector<int> members;               // batch indices
    int n_items = 0, max_n = 1;
    int threads_f = 64, threads_b = 64, smem_f = 0, smem_b = 0, ctas_f = 1, ctas_b = 1;
    grape::ScheduleParams* d_sched = nullptr;
    grape::QueueParams qf{}, qb{};
    int* d_counters = nullptr;              // head_f, head_b, done_f[Q], done_b[Q]
    size_t counter_bytes = 0;
  };
  std::vector<Queue> queues;
  int n_queued = 0, n_items = 0, queue_ctas = 0;
  bool refs_taken = false;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto e : events) cudaEventDestroy(e);
    for (auto s : streams) cudaStreamDestroy(s);
    if (origin) cudaStreamDestroy(origin);
    for (void* p : owned) cudaFree(p);
    if (refs_taken)
      for (grape_problem* P : probs) --P->batch_refs;
    refs_taken = false;
    probs.clear();
    exec = nullptr;
    graph = nullptr;
    events.clear();
    streams.clear();
    origin = nullptr;
    owned.clear();
  }
};

namespace {

template <typename T>
grape_status batch_upload(grape_batch* B, const std::vector<T>& host, T** dev) {
  void* ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(host.size(), 1) * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch queue)");
  B->owned.push_back(ptr);
  *dev = static_cast<T*>(ptr);
  if (!host.empty() && (e = cudaMemcpy(ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpy (batch queue)");
  return GRAPE_OK;
}

// A member's column teams are single CTAs in the forward and the fused backward sweep: its columns
// can be items of the work queue (members of the three-stage kind run their fused backward there).
bool queue_eligible(const grape_problem* P) {
  return !P->dense && !P->eig && P->fwd.CL == 1 && P->bwd.CL == 1 && (P->precision == 0 || P->precision == 1);
}

grape_status batch_build(grape_batch* B, int n_streams, int queue_ctas, const double* const* u_warm) {
  cudaError_t e;
  const int count = B->count;
  const int nsm = sm_count(B->device);
  // staging buffers (fixed addresses referenced by the graph)
  B->u_off.resize(count);
  B->g_off.resize(count);
  for (int i = 0; i < count; ++i) {
    B->u_off[i] = B->u_total;
    B->g_off[i] = B->g_total;
    B->u_total += (int64_t)B->probs[i]->K * B->probs[i]->N;
    B->g_total += (int64_t)B->probs[i]->K * B->probs[i]->N;
  }
  void* ptr = nullptr;
  const size_t bytes[3] = {(size_t)std::max<int64_t>(B->u_total, 1) * 8, (size_t)count * 8,
                           (size_t)std::max<int64_t>(B->g_total, 1) * 8};
  double** dst[3] = {&B->d_u, &B->d_cost, &B->d_grad};
  for (int k = 0; k < 3; ++k) {
    if ((e = cudaMalloc(&ptr, bytes[k])) != cudaSuccess) return cuda_fail(e, "cudaMalloc (batch staging)");
    B->owned.push_back(ptr);
    *dst[k] = static_cast<double*>(ptr);
    if ((e = cudaMemset(ptr, 0, bytes[k])) != cudaSuccess) return cuda_fail(e, "cudaMemset (batch staging)");
  }
  if ((e = cudaStreamCreateWithFlags(&B->origin, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  // one warm evaluation per problem outside the capture, at the caller's controls (else zero):
  // first launches set kernel attributes and constants (not stream work), and three-stage members
  // size their block buffers for this schedule
  for (int i = 0; i < count; ++i) {
    const size_t ub = (size_t)B->probs[i]->K * B->probs[i]->N * sizeof(double);
    if (u_warm && u_warm[i] && ub &&
        (e = cudaMemcpy(B->d_u + B->u_off[i], u_warm[i], ub, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpy (warm controls)");
  }
  // each warm evaluation is timed on its own (the split between the work queue and the lanes below)
  std::vector<double> t_warm(count, 0.0);
  {
    cudaEvent_t wa = nullptr, wb = nullptr;
    if ((e = cudaEventCreate(&wa)) != cudaSuccess || (e = cudaEventCreate(&wb)) != cudaSuccess) {
      if (wa) cudaEventDestroy(wa);
      return cuda_fail(e, "cudaEventCreate");
    }
    grape_status s = GRAPE_OK;
    for (int i = 0; i < count && !s; ++i) {
      grape_problem* P = B->probs[i];
      cudaEventRecord(wa, B->origin);
      if ((s = run_forward(P, B->d_u + B->u_off[i], true, B->origin))) break;
      if ((s = run_backward(P, B->origin))) break;
      cudaEventRecord(wb, B->origin);
      float ms = 0.0f;
      if ((e = cudaEventSynchronize(wb)) != cudaSuccess || (e = cudaEventElapsedTime(&ms, wa, wb)) != cudaSuccess)
        s = cuda_fail(e, "timing a warm evaluation");
      t_warm[i] = ms;
    }
    cudaEventDestroy(wa);
    cudaEventDestroy(wb);
    if (s) return s;
  }
  if ((e = cudaStreamSynchronize(B->origin)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  // work estimate of every member: Taylor terms of its sweep x union entries x columns
  std::vector<double> work(count), col_work(count);
  for (int i = 0; i < count; ++i) {
    grape_problem* P = B->probs[i];
    cudaMemset(P->d_err, 0, sizeof(int));
    if (P->eig) {   // one dense d x d product per step and column
      col_work[i] = (double)P->N * (double)P->dim * (double)P->dim;
      work[i] = col_work[i] * P->n;
      continue;
    }
    std::vector<int> m(P->N), sv(P->N);
    if ((e = cudaMemcpy(m.data(), P->d_ms_m, P->N * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(sv.data(), P->d_ms_s, P->N * sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "schedule download");
    double terms = 0.0;
    for (int n = 0; n < P->N; ++n) terms += (double)std::max(m[n], 0) * std::max(sv[n], 0);
    col_work[i] = std::max(terms, 1.0) * (double)P->nnz;
    work[i] = col_work[i] * P->n;
  }
  // queue membership (queue_ctas < 0: none) and the queues, one per bulk precision
  B->queued.assign(count, 0);
  double w_queue = 0.0;
  for (int i = 0; i < count; ++i) {
    if (queue_ctas >= 0 && queue_eligible(B->probs[i])) {
      B->queued[i] = 1;
      w_queue += work[i];
    }
  }
  for (int prec = 0; prec < 2; ++prec) {
    grape_batch::Queue q;
    q.precision = prec;
    for (int i = 0; i < count; ++i)
      if (B->queued[i] && B->probs[i]->precision == prec) q.members.push_back(i);
    if (!q.members.empty()) B->queues.push_back(std::move(q));
  }
  for (auto& q : B->queues) {
    const int Q = (int)q.members.size();
    std::vector<grape::ScheduleParams> sched(Q);
    std::vector<grape::SweepParams> fwd(Q), bwd(Q);
    std::vector<grape::FinalizeParams> fin(Q);
    std::vector<grape::GradReduceParams> red(Q);
    std::vector<int2> items;
    std::vector<double> item_cost;
    for (int j = 0; j < Q; ++j) {
      const int i = q.members[j];
      grape_problem* P = B->probs[i];
      double* u = B->d_u + B->u_off[i];
      sched[j] = schedule_params(P);
      sched[j].u = u;
      fwd[j] = sweep_params(P, P->fwd);
      fwd[j].u = u;
      bwd[j] = sweep_params(P, P->bwd);
      bwd[j].u = u;
      fin[j] = finalize_params(P, P->n);
      fin[j].u = u;
      fin[j].cost_out = B->d_cost + i;
      red[j] = grad_reduce_params(P, P->n);
      red[j].u = u;
      red[j].grad = B->d_grad + B->g_off[i];
      q.max_n = std::max(q.max_n, P->N);
      q.threads_f = std::max(q.threads_f, P->fwd.threads);
      q.threads_b = std::max(q.threads_b, P->bwd.threads);
      q.smem_f = std::max(q.smem_f, P->fwd.smem);
      q.smem_b = std::max(q.smem_b, P->bwd.smem);
      for (int c = 0; c < P->n; ++c) {
        items.push_back(make_int2(j, c));
        item_cost.push_back(col_work[i]);
      }
    }
    // longest first
    std::vector<int> idx(items.size());
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return item_cost[a] > item_cost[b]; });
    std::vector<int2> sorted(items.size());
    for (size_t k = 0; k < idx.size(); ++k) sorted[k] = items[idx[k]];
    q.n_items = (int)sorted.size();
    // CTAs: the queue's share of the work (the rest runs on the lanes) at the kernel's occupancy,
    // or the caller's count; never more than items
    const int occ_f = std::max(1, grape::queue_ctas_per_sm(q.precision, false, q.threads_f, q.smem_f));
    const int occ_b = std::max(1, grape::queue_ctas_per_sm(q.precision, true, q.threads_b, q.smem_b));
    // Automatic count: each queued member alone kept its n columns' CTAs busy for its warm time t, so
    // the queue holds sum(n_i t_i) CTA-ms of work; a lane member held about t x the SMs its teams
    // occupy.  Where the queued members carry under 5% of that, the lanes alone overlap them with the
    // large members and the queue is left out (measured on the 64-instance mix: 6.3 s on lanes
    // against 8.3-19.7 s with queues of 1-4 CTAs); otherwise the queue gets as many CTAs as it has
    // items, up to the whole GPU, and releases them as it drains.
    double q_cta_ms = 0.0, lane_sm_ms = 0.0;
    for (int i : q.members) q_cta_ms += (double)B->probs[i]->n * t_warm[i];
    for (int i = 0; i < count; ++i) {
      if (B->queued[i]) continue;
      const grape_problem* P = B->probs[i];
      const int team = P->eig ? 8 : std::max(P->fwd.CL, P->bwd.CL);
      const int sms = std::min(nsm, P->n * team * (P->bwd_mode == 3 ? 2 : 1));
      lane_sm_ms += t_warm[i] * sms;
    }
    const bool to_lanes = queue_ctas == 0 && q_cta_ms < 0.05 * lane_sm_ms;
    auto pick = [&](int occ) {
      if (queue_ctas > 0) return std::max(1, std::min(queue_ctas, q.n_items));
      return std::max(1, std::min(q.n_items, nsm * occ));
    };
    if (to_lanes) {
      for (int i : q.members) B->queued[i] = 0;
      q.members.clear();
      continue;
    }
    q.ctas_f = pick(occ_f);
    q.ctas_b = pick(occ_b);
    grape::SweepParams* d_fwd = nullptr;
    grape::SweepParams* d_bwd = nullptr;
    grape::FinalizeParams* d_fin = nullptr;
    grape::GradReduceParams* d_red = nullptr;
    int2* d_items = nullptr;
    grape_status st;
    if ((st = batch_upload(B, sched, &q.d_sched)) || (st = batch_upload(B, fwd, &d_fwd)) ||
        (st = batch_upload(B, bwd, &d_bwd)) || (st = batch_upload(B, fin, &d_fin)) ||
        (st = batch_upload(B, red, &d_red)) || (st = batch_upload(B, sorted, &d_items)))
      return st;
    std::vector<int> counters(2 + 2 * Q, 0);
    if ((st = batch_upload(B, counters, &q.d_counters))) return st;
    q.counter_bytes = counters.size() * sizeof(int);
    q.qf.sweep = d_fwd;
    q.qf.fin = d_fin;
    q.qf.items = d_items;
    q.qf.n_items = q.n_items;
    q.qf.head = q.d_counters;
    q.qf.done = q.d_counters + 2;
    q.qb.sweep = d_bwd;
    q.qb.red = d_red;
    q.qb.items = d_items;
    q.qb.n_items = q.n_items;
    q.qb.head = q.d_counters + 1;
    q.qb.done = q.d_counters + 2 + Q;
    B->n_queued += Q;
    B->n_items += q.n_items;
    B->queue_ctas = std::max(B->queue_ctas, std::max(q.ctas_f, q.ctas_b));
  }
  // the other members: longest first, greedy assignment to the least loaded lane; lane 0 also
  // carries the queues
  B->queues.erase(std::remove_if(B->queues.begin(), B->queues.end(),
                                 [](const grape_batch::Queue& q) { return q.members.empty(); }),
                  B->queues.end());
  w_queue = 0.0;
  for (int i = 0; i < count; ++i)
    if (B->queued[i]) w_queue += work[i];
  for (int i = 0; i < count; ++i)
    if (!B->queued[i]) B->order.push_back(i);
  std::stable_sort(B->order.begin(), B->order.end(), [&](int a, int b) { return work[a] > work[b]; });
  n_streams = std::max(1, std::min(n_streams, (int)B->order.size() + (B->queues.empty() ? 0 : 1)));
  std::vector<double> load(n_streams, 0.0);
  if (!B->queues.empty()) load[0] = w_queue;
  B->lane.assign(count, 0);
  for (int i : B->order) {
    const int j = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    B->lane[i] = j;
    load[j] += work[i];
  }
  B->streams.resize(n_streams);
  for (auto& s : B->streams)
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  B->events.resize(n_streams + 1);
  for (auto& ev : B->events)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
  // capture: fork onto the lanes, the queues on lane 0, every other member's sequence on its lane,
  // join back
  if ((e = cudaStreamBeginCapture(B->origin, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
    return cuda_fail(e, "cudaStreamBeginCapture");
  grape_status st = GRAPE_OK;
  cudaEventRecord(B->events[n_streams], B->origin);
  for (auto s : B->streams) cudaStreamWaitEvent(s, B->events[n_streams], 0);
  for (auto& q : B->queues) {
    cudaStream_t s = B->streams[0];
    if ((e = cudaMemsetAsync(q.d_counters, 0, q.counter_bytes, s)) != cudaSuccess) {
      st = cuda_fail(e, "cudaMemsetAsync (queue counters)");
      break;
    }
    if ((e = grape::launch_schedule_batch(q.d_sched, (int)q.members.size(), q.max_n, s)) != cudaSuccess) {
      st = cuda_fail(e, "launch k_schedule_batch");
      break;
    }
    if ((e = grape::launch_queue(q.qf, q.precision, false, q.ctas_f, q.threads_f, q.smem_f, s)) != cudaSuccess) {
      st = cuda_fail(e, "launch k_queue (forward)");
      break;
    }
    if ((e = grape::launch_queue(q.qb, q.precision, true, q.ctas_b, q.threads_b, q.smem_b, s)) != cudaSuccess) {
      st = cuda_fail(e, "launch k_queue (backward)");
      break;
    }
  }
  if (!st) {
    for (int i : B->order) {
      grape_problem* P = B->probs[i];
      cudaStream_t s = B->streams[B->lane[i]];
      if ((st = run_forward(P, B->d_u + B->u_off[i], true, s))) break;
      if ((st = run_backward(P, s))) break;
      if ((e = cudaMemcpyAsync(B->d_cost + i, P->d_cost, sizeof(double), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        st = cuda_fail(e, "cudaMemcpyAsync (batch cost)");
        break;
      }
      if (P->K > 0 && (e = cudaMemcpyAsync(B->d_grad + B->g_off[i], P->d_grad, (size_t)P->K * P->N * sizeof(double),
                                           cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
        st = cuda_fail(e, "cudaMemcpyAsync (batch grad)");
        break;
      }
    }
  }
  for (int j = 0; j < n_streams; ++j) {
    cudaEventRecord(B->events[j], B->streams[j]);
    cudaStreamWaitEvent(B->origin, B->events[j], 0);
  }
  e = cudaStreamEndCapture(B->origin, &B->graph);
  if (st) return st;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  if ((e = cudaGraphInstantiate(&B->exec, B->graph, 0)) != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return GRAPE_OK;
}

}  // namespace

extern "C" {

grape_status grape_batch_create(grape_problem* const* probs, int32_t count, int32_t n_streams, int32_t queue_ctas,
                                const double* const* u_warm, grape_batch** out) {
  if (!out) return fail(GRAPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!probs || count < 1) return fail(GRAPE_EINVAL, "need at least one problem");
  for (int i = 0; i < count; ++i) {
    if (!probs[i]) return fail(GRAPE_EINVAL, "NULL problem in batch");
    if (probs[i]->device != probs[0]->device) return fail(GRAPE_EINVAL, "batch problems must share one device");
    if (probs[i]->dense) return fail(GRAPE_EINVAL, "tensor-core problems are driven from the host and cannot join a batch");
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) return fail(GRAPE_EINVAL, "a problem appears twice in the batch");
  }
  DeviceGuard guard(probs[0]->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  grape_batch* B = new (std::nothrow) grape_batch();
  if (!B) return fail(GRAPE_ENOMEM, "host allocation failed");
  B->device = probs[0]->device;
  B->count = count;
  B->probs.assign(probs, probs + count);
  grape_status st;
  try {
    st = batch_build(B, n_streams <= 0 ? 8 : n_streams, queue_ctas, u_warm);
  } catch (...) {
    st = fail(GRAPE_ENOMEM, "host allocation failed");
  }
  if (!st) {   // the recording refers to the members' block buffers from now on
    for (grape_problem* P : B->probs) ++P->batch_refs;
    B->refs_taken = true;
  }
  if (st) {
    cudaDeviceSynchronize();
    B->release();
    delete B;
    return st;
  }
  *out = B;
  return GRAPE_OK;
}

void grape_batch_destroy(grape_batch* B) {
  if (!B) return;
  DeviceGuard guard(B->device);
  cudaDeviceSynchronize();
  B->release();
  delete B;
}

grape_status grape_batch_info(const grape_batch* B, grape_batch_info_t* out) {
  if (!B || !out) return fail(GRAPE_EINVAL, "NULL argument");
  out->members = B->count;
  out->queued = B->n_queued;
  out->queue_items = B->n_items;
  out->queue_ctas = B->queue_ctas;
  out->lanes = (int32_t)B->streams.size();
  out->lane_members = (int32_t)B->order.size();
  return GRAPE_OK;
}

grape_status grape_batch_cost_and_grad(grape_batch* B, const double* const* u, double* costs, double* const* grads,
                                       int32_t on_device, void* stream) {
  if (!B || !u || !costs) return fail(GRAPE_EINVAL, "NULL argument");
  DeviceGuard guard(B->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e;
  for (int i = 0; i < B->count; ++i) {
    const grape_problem* P = B->probs[i];
    const size_t n = (size_t)P->K * P->N;
    if (n == 0) continue;
    if (!u[i]) return fail(GRAPE_EINVAL, "NULL control array in batch");
    if ((e = cudaMemcpyAsync(B->d_u + B->u_off[i], u[i], n * 8, kin, st)) != cudaSuccess)
      return cuda_fail(e, "cudaMemcpyAsync (batch u)");
  }
  if ((e = cudaGraphLaunch(B->exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  if ((e = cudaMemcpyAsync(costs, B->d_cost, (size_t)B->count * 8, kout, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync (batch costs)");
  if (grads) {
    for (int i = 0; i < B->count; ++i) {
      const grape_problem* P = B->probs[i];
      const size_t n = (size_t)P->K * P->N;
      if (n == 0 || !grads[i]) continue;
      if ((e = cudaMemcpyAsync(grads[i], B->d_grad + B->g_off[i], n * 8, kout, st)) != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync (batch grad)");
    }
  }
  if (!on_device) {
    for (int i = 0; i < B->count; ++i) {
      grape_status s = read_error_word(B->probs[i], st);
      if (s) return s;
    }
  }
  return GRAPE_OK;
}

grape_status grape_optimize(grape_problem* P, double* u, int32_t n_iter, double eta, double* costs, int32_t on_device,
                            void* stream) {
  if (!P || (!u && P->K > 0) || !costs || n_iter < 1) return fail(GRAPE_EINVAL, "bad argument");
  if (!(eta > 0.0) || !std::isfinite(eta)) return fail(GRAPE_EINVAL, "eta must be finite and > 0");
  if (P->dense) return fail(GRAPE_EINVAL, "tensor-core problems are driven from the host and cannot be recorded");
  DeviceGuard guard(P->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  P->last_stream = st;
  cudaError_t e;
  const size_t ubytes = (size_t)P->K * P->N * sizeof(double);
  if (P->d_costs_cap < n_iter) {
    if (P->d_costs && (e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    // an optimizer-owned buffer, grown on demand (recording refers to it, so the graph is recorded again)
    void* pc = P->dalloc((size_t)n_iter * sizeof(double));
    if (!pc) return fail(GRAPE_ENOMEM, "device allocation failed");
    P->d_costs = static_cast<double*>(pc);
    P->d_costs_cap = n_iter;
    if (P->opt_exec) {
      cudaGraphExecDestroy(P->opt_exec);
      P->opt_exec = nullptr;
    }
  }
  if (!P->d_counter) {
    void* pc = P->dalloc(sizeof(int));
    if (!pc) return fail(GRAPE_ENOMEM, "device allocation failed");
    P->d_counter = static_cast<int*>(pc);
  }
  if (ubytes && (e = cudaMemcpyAsync(P->d_u, u, ubytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                     st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync (u)");
  if ((e = cudaMemsetAsync(P->d_counter, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  if (!P->opt_exec || P->opt_eta != eta) {
    if (P->opt_exec) {
      cudaGraphExecDestroy(P->opt_exec);
      P->opt_exec = nullptr;
    }
    // one evaluation outside the capture sets kernel attributes and constants (not stream work)
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    grape_status s2 = run_forward(P, P->d_u, true, cs);
    if (!s2) s2 = run_backward(P, cs);
    if (!s2 && (e = cudaStreamSynchronize(cs)) != cudaSuccess) s2 = cuda_fail(e, "cudaStreamSynchronize");
    cudaGraph_t g = nullptr;
    if (!s2 && (e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      s2 = cuda_fail(e, "cudaStreamBeginCapture");
    if (!s2) {
      s2 = run_forward(P, P->d_u, true, cs);
      if (!s2) s2 = run_backward(P, cs);
      if (!s2 && (e = grape::launch_sd_update(P->d_u, P->d_grad, (int64_t)P->K * P->N, eta, P->d_cost, P->d_costs,
                                              P->d_counter, P->d_costs_cap, cs)) != cudaSuccess)
        s2 = cuda_fail(e, "launch k_sd_update");
      const cudaError_t ee = cudaStreamEndCapture(cs, &g);
      if (!s2 && ee != cudaSuccess) s2 = cuda_fail(ee, "cudaStreamEndCapture");
    }
    if (!s2 && (e = cudaGraphInstantiate(&P->opt_exec, g, 0)) != cudaSuccess) s2 = cuda_fail(e, "cudaGraphInstantiate");
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (s2) return s2;
    P->opt_eta = eta;
  }
  // the stored sweep state belongs to the last evaluated iterate, not to the updated controls
  P->forward_done = false;
  for (int it = 0; it < n_iter; ++it)
    if ((e = cudaGraphLaunch(P->opt_exec, st)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  if (ubytes && (e = cudaMemcpyAsync(u, P->d_u, ubytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync (u out)");
  if ((e = cudaMemcpyAsync(costs, P->d_costs, (size_t)n_iter * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync (costs)");
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
  info->cluster = P->bwd.CL;
  info->cluster_forward = P->fwd.CL;
  info->ckpt_every = P->ckpt_every;
  info->smem_bytes = std::max(P->fwd.smem, P->bwd.smem);
  info->total_terms = -1;
  info->max_norm = -1.0;
  info->backward_mode = P->bwd_mode;
  info->propagator = P->eig ? GRAPE_PROP_EIG : GRAPE_PROP_TAYLOR;
  info->fused_fallback = -1;
  if (P->bwd_mode == 3) {
    info->grad_cluster = P->grd.CL;
    info->block_steps = P->steps_per_block;
    if (P->evaluated) {
      DeviceGuard guard(P->device);
      int flag = 0;
      cudaStreamSynchronize(P->last_stream);
      if (cudaMemcpy(&flag, P->d_plan_flag, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(GRAPE_ECUDA, "cudaMemcpy (plan flag)");
      info->fused_fallback = flag;
    }
  }
  if (P->evaluated && !P->eig) {
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

grape_status grape_set_kernel_tracing(grape_problem* P, int32_t enable) {
  if (!P) return fail(GRAPE_EINVAL, "NULL problem");
  P->tracing = enable != 0;
  P->tr_used = 0;
  return GRAPE_OK;
}

grape_status grape_kernel_times(grape_problem* P, grape_kernel_times_t* out) {
  if (!P || !out) return fail(GRAPE_EINVAL, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  DeviceGuard guard(P->device);
  if (!guard.ok) return fail(GRAPE_ECUDA, "cudaSetDevice failed");
  for (size_t i = 0; i < P->tr_used; ++i) {
    cudaError_t e = cudaEventSynchronize(P->tr_events[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
    float ms = 0.0f;
    if ((e = cudaEventElapsedTime(&ms, P->tr_events[2 * i], P->tr_events[2 * i + 1])) != cudaSuccess)
      return cuda_fail(e, "cudaEventElapsedTime");
    out->launches[P->tr_kind[i]] += 1;
    out->ms[P->tr_kind[i]] += ms;
  }
  P->tr_used = 0;
  return GRAPE_OK;
}

grape_status grape_step_schedule(grape_problem* P, int32_t* m, int32_t* s, double* norm1) {
  if (!P) return fail(GRAPE_EINVAL, "NULL problem");
  if (P->eig) return fail(GRAPE_EINVAL, "GRAPE_PROP_EIG problems have no Taylor schedule");
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
