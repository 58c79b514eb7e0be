// Eigendecomposition variant of the HG evaluation (App. F): device buffers and launchers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace grape {

constexpr int kEigMaxDim = 96;   // the step matrix and its eigenvector block live in shared memory

struct EigCtx {
  int d, n, N, K;
  int sweep_cl;           // CTAs per column (one cluster) in the forward and backward sweeps
  int step0, nsteps;      // steps [step0, step0 + nsteps) of one launch of the per-step kernels and
                          // of the forward sweep (the backward kernels take all N steps)
  double dt, w_fid, w_forbid, w_tint;
  const double2* H0;      // d x d dense drift, row-major
  const double2* Hk;      // K x d x d dense controls, row-major (Hermitian)
  const double* u;        // K x N controls
  const int* cp_ptr;      // d + 1: column b of the union pattern of the controls holds rows
  const int* cp_row;      //   cp_row[cp_ptr[b] .. cp_ptr[b + 1]) (ascending)
  double* lam;            // N x d eigenvalues of H_n
  double2* V;             // N x d x d eigenvectors (column c of V_n is the c-th eigenvector)
  double2* Vt;            // N x d x d transposed copy (Vt_n[c][i] = V_n[i][c])
  double2* U;             // N x d x d step propagators (Householder vectors of the step until they are replaced)
  double* htau;           // N x d Householder scalars
  double* tri_a;          // N x d diagonal of the tridiagonal form
  double2* tri_t;         // N x d super-diagonal t_i = T_{i,i+1} (complex)
  double2* phase;         // N x d diagonal phases that make the tridiagonal real
  int rot_cap;            // recorded plane rotations per step (capacity)
  int* rot_i;             // N x rot_cap rotation index i (columns i, i+1)
  double2* rot_cs;        // N x rot_cap (c, s)
  int* rot_n;             // N rotations recorded
  const double2* psi0;    // d x n column-major
  const double2* target;  // d x n column-major
  const double* omega;    // d or nullptr
  double2* psi_hist;      // (N + 1) x n x d: psi_s, s = 0..N
  double2* chi_hist;      // (N + 1) x n x d: chi_s, s = 1..N
  double2* xs;            // N x 2 x n x d: V_s^+ psi_{s-1} and V_s^+ chi_s (gradient scratch)
  double2* part_g;        // n
  double* part_c2;        // n
  double2* part_g3;       // n x N (C3 overlaps), or nullptr
  const double2* g_final; // after the finalize
  const double2* g3;      // N after the finalize
  double* part_grad;      // N x K
  int* err;
};

int eig_step_smem(int d);
int eig_qr_smem(int d);
int eig_rotate_smem(int d);
int eig_grad_smem(int d, int K);
cudaError_t eig_prepare(int d, int K);
// Eigenpairs and propagators of steps [c.step0, c.step0 + c.nsteps) (independent across steps).
cudaError_t eig_propagators(const EigCtx& c, cudaStream_t st);
// Forward sweep over steps [c.step0, c.step0 + c.nsteps); launches of one sweep follow each other.
cudaError_t eig_forward_sweep(const EigCtx& c, cudaStream_t st);
cudaError_t eig_backward(const EigCtx& c, cudaStream_t st);

}  // namespace grape
