// Internal declarations shared by the host library and the CUDA kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace grape {

constexpr int kMaxControls = 32;
constexpr int kMaxTaylor = 60;       // m_max cap (Sec. III.B leaves it open)
constexpr int kMaxCluster = 16;
constexpr int kOwnerShift = 20;      // column encoding: bit 31 = entry carries control terms,
constexpr uint32_t kLocalMask = (1u << kOwnerShift) - 1u;   // bits 20..27 owner CTA, bits 0..19 local row
constexpr uint32_t kCtrlBit = 1u << 31;
constexpr uint32_t kImagBBit = 1u << 30;   // off-diagonal entry whose B_ij is imaginary (every H_ij term real)
constexpr uint32_t kRealBBit = 1u << 29;   // off-diagonal entry whose B_ij is real (every H_ij term imaginary)

// Device error word values (same numbering as grape_status).
constexpr int kErrTol = 4;
constexpr int kErrTimeout = 5;
constexpr int kErrNonFinite = 8;
constexpr int kErrEig = 9;

// Everything a sweep kernel needs; passed by value.
struct SweepParams {
  // problem
  int dim, K, N, n_states, CL, R;      // CL = CTAs per column team, R = rows per CTA
  double dt;
  double w_fid, w_forbid, w_amp, w_tint;
  int ckpt_every;                      // 0 = no checkpoints
  int n_ckpt;                          // number of stored checkpoints
  int m_cap;
  // union pattern (global)
  int diag_first;                      // 1: every diagonal H_ii is real and, where present, is the
                                       // first entry of its row (B_ii = -i dt H_ii / s is imaginary).
                                       // Rows continue with the kImagBBit entries, then the kRealBBit
                                       // entries, then the rest; each segment in ascending columns.
  const int64_t* rowptr;               // dim + 1
  const uint32_t* colenc;              // nnz, per CL-partition encoding (owner, local, ctrl bit)
  const double2* h0v;                  // nnz drift values on the union pattern
  // per-control contribution lists: entries of control k are [cptr[k], cptr[k+1]) sorted by entry
  const int* cptr;                     // K + 1
  const int* cidx;                     // global union-entry index
  const double2* cval;                 // value of h_k at that entry
  const int* cslice;                   // [(k * CL + rank) * 2 + {0,1}]: range of control k inside rank's rows
  // controls and schedule
  const double* u;                     // K x N row-major (device)
  const int* ms_m;                     // N
  const int* ms_s;                     // N
  // states
  const double2* psi0;                 // d x n column-major
  const double2* target;               // d x n
  const double* omega;                 // d or nullptr
  double2* psiN;                       // d x n
  double2* ckpt;                       // n_ckpt x n x d
  // reductions
  double2* part_g;                     // n_teams * CL
  double* part_c2;                     // n_teams * CL
  double* part_grad;                   // (n_teams * CL) x N x K
  const double2* g_final;              // device scalar g (after the forward finalize)
  double2* part_g3;                    // (n_teams * CL) x N: per-step overlap partials (C3)
  const double2* g3;                   // N per-step overlaps g_n (after the finalize)
  // scratch for buffers that do not fit in shared memory (per CTA slices)
  double2* scratch;
  int64_t scratch_stride;              // doubles2 per CTA
  // shared-memory plan (see make_layout) and scratch offsets (in double2 units) of the
  // buffers that are not in shared memory
  int in_smem, m_smem;
  int64_t scr_vals, scr_W, scr_Wb, scr_wslot;
  int max_nnz_loc;
  // entry-major control contributions (for assembling H_n on the union pattern)
  const int* ectr_ptr;                 // nnz + 1
  const int* ectr_k;
  const double2* ectr_val;
  int* err;                            // device error word
  // three-stage backward: k_costate (costate chain) and k_gradient (per-step gradient) work on the
  // block of steps [n_begin, n_end); k_plan decides once per evaluation whether they run
  int n_begin, n_end;
  double2* chi_io;                     // d x n: the costate carried from one k_costate launch to the next
  void* hbuf;                          // Horner vectors of the block, bulk type: [term][column][row]
  int64_t hbuf_terms;                  // capacity of hbuf in terms
  const int* plan_flag;                // 0: the three-stage kernels run; 1: the fused k_backward runs instead
  int gate_on_flag;                    // k_backward: 1 = run only when *plan_flag != 0 (the fallback)
  // segment recompute (three-stage backward, checkpoints every seg_M > 1 steps): states psi_n of the
  // segment [j M, (j+1) M) live in slot j % 2 of seg (2 x seg_M x n x dim); k_forward with
  // recompute = 1 runs steps [n_begin, n_end) from rec_src (psi_{n_begin}) and fills the slot
  double2* seg;
  int seg_M;
  int recompute;
  const double2* rec_src;
};

// Block plan of the three-stage backward: per block of S steps the Horner vectors of every term must
// fit in the block's buffer; if any block's sum of m_n s_n exceeds the capacity the flag is set and
// the fused one-team backward runs instead (both paths are queued, each returns at once when the
// flag says the other one runs).
struct PlanParams {
  int N, steps_per_block;
  int64_t cap_terms;
  const int* ms_m;
  const int* ms_s;
  int* flag;
};

struct ScheduleParams {
  int dim, K, N;
  double dt;
  const int64_t* rowptr;
  const double2* h0v;
  const int* ectr_ptr;
  const int* ectr_k;
  const double2* ectr_val;
  const double* u;
  const double* table;                 // s_cap x m_cap breakpoints X[s-1][m-1] (largest feasible x), < 0 = never
  const double* table_smax;            // s_cap: max over m of X
  int m_cap, s_cap;
  double b_cap;                        // > 0: only pairs with ||B||_1 = x / s <= b_cap
  int* ms_m;
  int* ms_s;
  double* norm1;
  int* err;
};

struct FinalizeParams {
  int n_parts, n_states, N, K;
  double w_fid, w_forbid, w_amp, w_tint;
  const double2* part_g3;              // n_parts x N (C3), or nullptr
  double2* g3_out;                     // N
  const double2* part_g;
  const double* part_c2;
  const double* u;
  double2* g_out;
  double* cost_out;
  double* parts_out;                   // [C1, C2, C_amp, |g|, C3]
};

struct GradReduceParams {
  int n_parts, N, K;
  int n_parts_alt;                     // parts summed when *plan_flag != 0 (the fused fallback ran)
  const int* plan_flag;                // nullptr: always n_parts
  double w_amp;
  const double* part_grad;
  const double* u;
  double* grad;                        // K x N row-major
};

// Batch work queue (k_queue): (problem, column) items, longest first, over problems whose column
// teams are single CTAs.  head and done[] start at zero for every launch.
struct QueueParams {
  const SweepParams* sweep;            // per problem: its forward or fused-backward sweep (CL = 1)
  const FinalizeParams* fin;           // forward queue: per problem, run by the CTA finishing its last column
  const GradReduceParams* red;         // backward queue: the same for the gradient reduction
  const int2* items;                   // (problem, column)
  int n_items;
  int* head;                           // next item to take
  int* done;                           // per problem: columns finished
};

// Dynamic shared-memory layout of the sweep kernels (byte offsets).  Exchange buffers,
// per-row states and the local pattern always live in shared memory; the drift-plus-control
// values (vals), the per-entry gradient accumulators (W) and the first m_smem Horner slots
// (wslot) live there when they fit, else in the CTA's global scratch slice.
struct SmemLayout {
  int xbuf;          // exchange buffers: nchains x 2 x R bulk complex
  int psi, chi, inc; // R double2 each (chi only in the backward sweep)
  int vals, W, Wb, wslot;
  int lrow, lcol;    // R + 1 ints, max_nnz_loc uints
  int total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// in_smem bit 0: vals, bit 1: W, bit 2: Wb (per-substep compensated staging of W, staged = true for the
// compensated FP32 bulk, 16 bytes per entry); m_smem = Horner slots kept in
// shared memory; cplx_bytes = 16 (one bulk complex: double2, or float4 for the compensated FP32 bulk).
__host__ __device__ inline SmemLayout make_layout(bool backward, int R, int max_nnz_loc, int in_smem, int m_smem,
                                                  int cplx_bytes, bool staged) {
  SmemLayout L;
  const int nchains = backward ? 3 : 1;
  int off = 0;
  L.xbuf = off; off += align16(nchains * 2 * R * cplx_bytes);
  L.psi = off;  off += align16(R * 16);
  L.chi = -1;
  if (backward) { L.chi = off; off += align16(R * 16); }
  L.inc = off;  off += align16(R * 16);
  L.vals = -1; L.W = -1; L.Wb = -1; L.wslot = -1;
  if (in_smem & 1) { L.vals = off; off += align16(max_nnz_loc * cplx_bytes); }
  if (backward && (in_smem & 2)) { L.W = off; off += align16(max_nnz_loc * 16); }
  if (backward && staged && (in_smem & 4)) { L.Wb = off; off += align16(max_nnz_loc * 16); }
  if (backward && m_smem > 0) { L.wslot = off; off += align16(m_smem * R * cplx_bytes); }
  L.lrow = off; off += align16((R + 1) * 4);
  L.lcol = off; off += align16(max_nnz_loc * 4);
  L.total = off;
  return L;
}

// Layout of k_gradient (byte offsets): the x chain's two exchange buffers, psi^(l), the increment,
// then vals (in_smem bit 0) and W (bit 1, FP64 accumulators per local entry) and, for the compensated FP32
// bulk, the compensated staging of W (bit 2, 16 bytes per entry), then the local pattern.
__host__ __device__ inline SmemLayout make_glayout(int R, int max_nnz_loc, int in_smem, int cplx_bytes, bool staged) {
  SmemLayout L;
  int off = 0;
  L.xbuf = off; off += align16(2 * R * cplx_bytes);
  L.psi = off;  off += align16(R * 16);
  L.chi = -1;
  L.inc = off;  off += align16(R * 16);
  L.vals = -1; L.W = -1; L.Wb = -1; L.wslot = -1;
  if (in_smem & 1) { L.vals = off; off += align16(max_nnz_loc * cplx_bytes); }
  if (in_smem & 2) { L.W = off; off += align16(max_nnz_loc * 16); }
  if (staged && (in_smem & 4)) { L.Wb = off; off += align16(max_nnz_loc * 16); }
  L.lrow = off; off += align16((R + 1) * 4);
  L.lcol = off; off += align16(max_nnz_loc * 4);
  L.total = off;
  return L;
}

// Launchers (grape_kernels.cu).  Return cudaGetLastError() of the launch.
cudaError_t launch_schedule(const ScheduleParams& p, cudaStream_t st);
cudaError_t launch_forward(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st);
cudaError_t launch_backward(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st);
cudaError_t launch_plan(const PlanParams& p, cudaStream_t st);
// priority: launch priority of the costate chain (the critical path), e.g. the device's greatest
cudaError_t launch_costate(const SweepParams& p, int precision, int smem_bytes, int threads, int priority,
                           cudaStream_t st);
cudaError_t launch_gradient(const SweepParams& p, int precision, int smem_bytes, int threads, cudaStream_t st);
cudaError_t launch_finalize(const FinalizeParams& p, cudaStream_t st);
cudaError_t launch_grad_reduce(const GradReduceParams& p, cudaStream_t st);
cudaError_t check_nonfinite_u(const double* u, int64_t count, int* err, cudaStream_t st);
// Batch: the schedules of `count` problems (device array ps, max_n = their largest N) in one launch,
// and the persistent work-queue sweeps (precision 0 FP64, 1 compensated FP32 bulk).
cudaError_t launch_schedule_batch(const ScheduleParams* ps, int count, int max_n, cudaStream_t st);
int queue_ctas_per_sm(int precision, bool backward, int threads, int smem_bytes);
cudaError_t launch_queue(const QueueParams& q, int precision, bool backward, int ctas, int threads, int smem_bytes,
                         cudaStream_t st);
cudaError_t launch_sd_update(double* u, const double* grad, int64_t count, double eta, const double* cost, double* costs,
                             int* counter, int max_count, cudaStream_t st);
int max_dynamic_smem(int device);

}  // namespace grape
