// Discrete elastic energy of a caller-owned DOF array without any device allocation.
//
// For callers that cannot call cudaMalloc: applications whose device memory is owned by
// another framework's pool or arena, code that must not allocate (and so must not risk an
// allocation failure or the implicit synchronisation of cudaMalloc/cudaFree) once it has
// started time stepping, and embedded or real-time hosts that reserve all device memory
// up front. They pass their own inputs and output; the only scratch is the per-element
// energy array below, a file-scope device array that every GPU which loads this library
// keeps until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ader_lts.h"

namespace {

static __device__ __align__(256) double g_noalloc_elem_energy[LTS_NOALLOC_MAX_ELEMENTS];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// 1/2 rho |v|^2 + 1/2 sigma : C^-1 sigma summed over the modes of one element, times |det J|
// (orthonormal basis: the L2 norm on an element is |det J| times the coefficient norm).
__global__ void k_elem_energy(const float* __restrict__ dofs, const double* __restrict__ mat, int64_t n_elem,
                              int nq, int nb, double* __restrict__ scratch) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_elem) return;
  const float* q = dofs + k * nq * nb;
  const double lam = mat[4 * k], mu = mat[4 * k + 1], rho = mat[4 * k + 2], detj = mat[4 * k + 3];
  const double cmp = lam / (2.0 * mu * (3.0 * lam + 2.0 * mu));
  double e = 0.0;
  for (int b = 0; b < nb; ++b) {
    double s[6], v[3];
    for (int r = 0; r < 6; ++r) s[r] = q[r * nb + b];
    for (int r = 0; r < 3; ++r) v[r] = q[(6 + r) * nb + b];
    const double tr = s[0] + s[1] + s[2];
    const double ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] + 2.0 * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
    e += 0.5 * (ss / (2.0 * mu) - cmp * tr * tr) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  }
  scratch[k] = detj * e;
}

// One block sums the per-element energies in a fixed order (deterministic).
__global__ void k_sum(const double* __restrict__ scratch, int64_t n, double* __restrict__ out) {
  __shared__ double red[1024];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += scratch[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Device address of the scratch array on the current device, looked up once per device.
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_elem_energy);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int lts_energy_noalloc(int order, int n_mech, const float* dofs, const double* mat, int64_t n_elem,
                                  double* energy, void* cuda_stream) {
  if (order < 3 || order > 5 || (n_mech != 0 && n_mech != 3) || !dofs || !mat || !energy) return LTS_ERR_ARG;
  if (n_elem <= 0 || n_elem > LTS_NOALLOC_MAX_ELEMENTS) return LTS_ERR_ARG;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return LTS_ERR_CUDA;
  const int nb = order * (order + 1) * (order + 2) / 6;
  const int nq = 9 + 6 * n_mech;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int threads = 256;
  const unsigned blocks = (unsigned)((n_elem + threads - 1) / threads);
  k_elem_energy<<<blocks, threads, 0, st>>>(dofs, mat, n_elem, nq, nb, scratch);
  k_sum<<<1, 1024, 0, st>>>(scratch, n_elem, energy);
  return cudaGetLastError() == cudaSuccess ? LTS_OK : LTS_ERR_CUDA;
}
