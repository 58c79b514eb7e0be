// grape_taylor_step_noalloc: one propagation step that needs no device allocation.
//
// The paper has no counterpart to this entry point; it exists for callers that
// cannot allocate device memory.  Its working memory (two Taylor-term buffers and
// one accumulator per column) is a fixed array compiled into this library and
// resident on every GPU that loads the library until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/grape_hg.h"
#include "grape_internal.h"

namespace grape {
void set_last_error(const std::string& msg);   // defined in grape_host.cpp
}

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
constexpr size_t kNoAllocScratchElems = kNoAllocScratchBytes / sizeof(double2);
// Largest substep count accepted: the same cap as the (m, s) table of the descriptor path.  It bounds
// one call's sequential work (s * m sparse products per column in one CTA).
constexpr int32_t kNoAllocMaxS = 4096;

// Shared by every call on a device; keeps whatever the last call left in it.
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double2* g_scratch_addr[kMaxDevices] = {nullptr};

// psi_out = (e^{B}_m)^s psi_in with B = -i dt H / s: the forward sweep's inner loop for one step
// (b_q = (B/q) b_{q-1}, summed per substep), one CTA per column, the three working vectors of a
// column in the static scratch array.  Every buffer is written before it is read, so nothing in
// the scratch needs to start at zero.  Each row's entry range is clamped to [0, nnz) and column
// indices outside [0, dim) are skipped, so a malformed rowptr or colind cannot make the kernel read
// outside the caller's arrays.
__global__ void __launch_bounds__(256) k_taylor_step_noalloc(int dim, int64_t nnz, const int64_t* __restrict__ rowptr,
                                                             const int32_t* __restrict__ colind,
                                                             const double2* __restrict__ vals, double scale, int m,
                                                             int s, const double2* psi_in, double2* psi_out,
                                                             double2* scratch) {
  const int h = blockIdx.x;
  double2* T0 = scratch + (int64_t)h * 3 * dim;
  double2* T1 = T0 + dim;
  double2* acc = T1 + dim;
  for (int i = threadIdx.x; i < dim; i += blockDim.x) acc[i] = psi_in[(int64_t)h * dim + i];
  __syncthreads();
  for (int l = 0; l < s; ++l) {
    for (int i = threadIdx.x; i < dim; i += blockDim.x) T0[i] = acc[i];
    __syncthreads();
    for (int q = 1; q <= m; ++q) {
      const double2* src = (q & 1) ? T0 : T1;
      double2* dst = (q & 1) ? T1 : T0;
      const double iq = 1.0 / q;
      for (int i = threadIdx.x; i < dim; i += blockDim.x) {
        double2 y = make_double2(0.0, 0.0);
        const int64_t ea = max(rowptr[i], (int64_t)0), eb = min(rowptr[i + 1], nnz);
        for (int64_t e = ea; e < eb; ++e) {
          const double2 v = vals[e];
          const double2 b = make_double2(scale * v.y, -scale * v.x);   // -i (dt/s) H_ij
          const int32_t j = colind[e];
          if ((uint32_t)j >= (uint32_t)dim) continue;   // out-of-range column: entry ignored
          const double2 x = src[j];
          y.x = fma(b.x, x.x, y.x);
          y.x = fma(-b.y, x.y, y.x);
          y.y = fma(b.x, x.y, y.y);
          y.y = fma(b.y, x.x, y.y);
        }
        y.x *= iq;
        y.y *= iq;
        dst[i] = y;
        double2 a = acc[i];
        a.x += y.x;
        a.y += y.y;
        acc[i] = a;
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < dim; i += blockDim.x) psi_out[(int64_t)h * dim + i] = acc[i];
}

grape_status noalloc_fail(grape_status st, const std::string& msg) {
  grape::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" grape_status grape_taylor_step_noalloc(int64_t dim, int64_t nnz, int32_t n_states, const int64_t* rowptr,
                                                  const int32_t* colind, const double* values, double dt, int32_t m,
                                                  int32_t s, const double* psi_in, double* psi_out, void* stream) {
  if (dim < 1 || dim >= (int64_t(1) << 31) || n_states < 1)
    return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: dim and n_states must be >= 1");
  if (nnz < 0) return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: nnz must be >= 0");
  if (m < 1 || m > grape::kMaxTaylor || s < 1 || s > kNoAllocMaxS)
    return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: need 1 <= m <= 60 and 1 <= s <= 4096");
  if (!(dt > 0.0) || !std::isfinite(dt)) return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: dt must be finite and > 0");
  if (!rowptr || !colind || !values || !psi_in || !psi_out)
    return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: NULL pointer");
  const size_t need = size_t(3) * size_t(dim) * size_t(n_states);
  if (need > kNoAllocScratchElems)
    return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: 3 * dim * n_states complex numbers exceed the "
                                      "16 MiB static scratch (at most 349525 = 16 MiB / 48 B)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(GRAPE_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(GRAPE_EINVAL, "grape_taylor_step_noalloc: device ordinal >= 64");
  double2* scratch = nullptr;
  {
    // First call on this device (which must be current): look up the device address of the static
    // array once.  In host code the array's name is only a host-side stand-in.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return noalloc_fail(GRAPE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = static_cast<double2*>(ptr);
    }
    scratch = g_scratch_addr[dev];
  }
  k_taylor_step_noalloc<<<n_states, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      (int)dim, nnz, rowptr, colind, reinterpret_cast<const double2*>(values), dt / s, m, s,
      reinterpret_cast<const double2*>(psi_in), reinterpret_cast<double2*>(psi_out), scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(GRAPE_ECUDA, std::string("launch k_taylor_step_noalloc: ") + cudaGetErrorString(e));
  return GRAPE_OK;
}
