// Dense-operator (tensor-core) variant of the HG evaluation: host-side driver interface.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace grape {

struct DenseCtx {
  CUtensorMap tm[8];        // TMA views of brh, brl, bih, bil, xh, xl, xh2, xl2 (dense_make_maps)
  int d, n, N, K, ksplit;
  int x_rows;               // rows allocated in xh / xl (>= 4 n, >= 64, a multiple of 16)
  int bf16;                 // operand pairs are bf16 (GRAPE_TC_BF16), else fp16 (GRAPE_TC_FP16)
  double dt, w_fid, w_forbid, w_tint;
  int ckpt_every, n_ckpt;
  double inv_fact[62];
  // operator of the current step (FP16 hi/lo of Br and Bi, d x d row-major) and work blocks
  __half *brh, *brl, *bih, *bil;
  __half *xh, *xl;          // x_rows x d: real columns of up to 2 n complex columns (tiled storage)
  __half *xh2, *xl2;        // the second X buffer pair: a product reads one and writes the other
  float2* y;                // d x 2n complex, column-major
  double2 *psi, *chi, *inc; // d x n
  float2* wslot;            // m_cap x d x n Horner vectors (FP32)
  float2* xcur;             // d x n current x_p (FP32)
  double2* W;               // control entries
  int nce;
  const int *ce_row, *ce_col;
  const int *cptr, *cce;    // per-control contribution lists -> control-entry index
  const double2* cval;
  // union pattern and values
  const int64_t* rowptr;
  const int* ucol;
  const double2* h0v;
  const int *ectr_ptr, *ectr_k;
  const double2* ectr_val;
  const double* u;
  const double2 *psi0, *target;
  const double* omega;
  double2 *psiN, *ckpt;
  double2* part_g;          // 1
  double* part_c2;          // 1
  double* c2acc;            // 1
  const double2* g_final;
  double2* part_g3;         // N per-step overlaps (C3) written by the forward sweep
  const double2* g3;        // N, after the finalize
  double* part_grad;        // N x K
  int* err;
};

int dense_apply_smem(int nreal);
// Tensor maps of the operator and X buffers (after they are allocated); cudaErrorNotSupported if the
// driver offers no tensor-map encoder.
cudaError_t dense_make_maps(DenseCtx& c);
cudaError_t dense_prepare();
int dense_choose_ksplit(int d);
cudaError_t dense_forward(const DenseCtx& c, const int* m_host, const int* s_host, cudaStream_t st);
cudaError_t dense_backward(const DenseCtx& c, const int* m_host, const int* s_host, cudaStream_t st);

}  // namespace grape
