// memd_static.cu -- memd_field_energy_static: the field-energy reduction for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside another
// framework's allocator or memory pool, a host that has pre-reserved every
// byte of device memory for its own arena, or a real-time loop that must not
// risk an allocation failing or blocking the device.  For them this entry
// point does the same reduction as the electric and magnetic terms of
// memd_energy, on device arrays the caller owns, without any allocation: its
// per-block partial sums live in a fixed file-scope device array.
//
// The array (MEMD_STATIC_MAX_BLOCKS x 2 doubles, 1 MiB) is part of the
// library image, so every GPU that loads the library holds it until the
// process exits.  Every call shares it: the partial sums are overwritten by
// each call (nothing needs to start at zero), and two calls whose kernels
// overlap on the GPU race on it, so the caller must serialise them (one
// stream, or events).
#include <mutex>

#include "memd.h"
#include "memd_internal.cuh"

namespace memd {
namespace {

constexpr int kThreads = 256;
constexpr int kSitesPerBlock = MEMD_STATIC_SITES_PER_BLOCK;
constexpr int kMaxBlocks = MEMD_STATIC_MAX_BLOCKS;

// partial sums: [0, kMaxBlocks) electric, [kMaxBlocks, 2 kMaxBlocks) magnetic
static __device__ __align__(256) double g_static_partials[2 * kMaxBlocks];

__device__ inline double block_sum(double x, double* sh) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = x;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)(blockDim.x >> 5); ++t) r += sh[t];
  __syncthreads();
  return r;
}

// Block b sums sites [b S, (b+1) S) of a^3-free electric D^2 ie / 2 and
// magnetic B (B - cB circ E) terms into part[b] and part[nb + b].
template <typename T>
__global__ void __launch_bounds__(kThreads)
    k_energy_partials(Mesh m, const T* __restrict__ D, const T* __restrict__ B,
                      const T* __restrict__ ie, double cB, double* __restrict__ part, int nb) {
  __shared__ double sh[kThreads / 32];
  const int64_t V = m.V;
  double el = 0.0, mag = 0.0;
  const int64_t v0 = (int64_t)blockIdx.x * kSitesPerBlock;
  for (int64_t v = v0 + threadIdx.x; v < V && v < v0 + kSitesPerBlock; v += kThreads) {
    const int i = (int)(v % m.n[0]);
    const int64_t r = v / m.n[0];
    const int j = (int)(r % m.n[1]);
    const int k = (int)(r / m.n[1]);
    const int ip = (i + 1 == m.n[0]) ? 0 : i + 1;
    const int jp = (j + 1 == m.n[1]) ? 0 : j + 1;
    const int kp = (k + 1 == m.n[2]) ? 0 : k + 1;
    const int64_t vx = vindex(m, ip, j, k), vy = vindex(m, i, jp, k), vz = vindex(m, i, j, kp);
    double E[3], Ex_[3], Ey_[3], Ez_[3];
    for (int d = 0; d < 3; ++d) {
      const double dd = (double)D[d * V + v], ii = (double)ie[d * V + v];
      E[d] = dd * ii;
      el += 0.5 * dd * dd * ii;
      Ex_[d] = (double)D[d * V + vx] * (double)ie[d * V + vx];
      Ey_[d] = (double)D[d * V + vy] * (double)ie[d * V + vy];
      Ez_[d] = (double)D[d * V + vz] * (double)ie[d * V + vz];
    }
    const double cx = ((E[1] + Ey_[2]) - Ez_[1]) - E[2];
    const double cy = ((E[2] + Ez_[0]) - Ex_[2]) - E[0];
    const double cz = ((E[0] + Ex_[1]) - Ey_[0]) - E[1];
    const double bx = (double)B[v], by = (double)B[V + v], bz = (double)B[2 * V + v];
    mag += bx * (bx - cB * cx) + by * (by - cB * cy) + bz * (bz - cB * cz);
  }
  const double s1 = block_sum(el, sh);
  const double s2 = block_sum(mag, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s1;
    part[nb + blockIdx.x] = s2;
  }
}

// out[0] = a^3 sum(el), out[1] = (c^2 a^3 / 2) sum(mag), in fixed block order
__global__ void __launch_bounds__(kThreads)
    k_energy_finish(const double* __restrict__ part, int nb, double a3, double half_c2_a3,
                    double* __restrict__ out) {
  __shared__ double sh[kThreads / 32];
  double s1 = 0.0, s2 = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    s1 += part[b];
    s2 += part[nb + b];
  }
  s1 = block_sum(s1, sh);
  s2 = block_sum(s2, sh);
  if (threadIdx.x == 0) {
    out[0] = s1 * a3;
    out[1] = s2 * half_c2_a3;
  }
}

// device address of the scratch array, looked up once per device with that
// device current and kept for the life of the process (a device reset after
// the first call would leave it stale: not supported)
std::mutex g_mu;
double* g_addr[64] = {nullptr};

}  // namespace
}  // namespace memd

extern "C" memd_status memd_field_energy_static(const int32_t mesh[3], double a, double c_light,
                                                double dt, int32_t precision, const void* D,
                                                const void* B, const void* inv_eps,
                                                double* out2, void* cuda_stream) {
  using namespace memd;
  if (!mesh || !D || !B || !inv_eps || !out2) return MEMD_ERR_INVALID;
  if (precision != MEMD_FP32 && precision != MEMD_FP64) return MEMD_ERR_INVALID;
  if (!(a > 0.0) || !(c_light > 0.0) || !(dt > 0.0)) return MEMD_ERR_INVALID;
  // each edge, then the vertex count, is bounded before it can wrap: a
  // wrapped count would pass the limit and send the kernel far outside the
  // caller's arrays
  int64_t V = 1;
  for (int d = 0; d < 3; ++d) {
    if (mesh[d] < 2 || (int64_t)mesh[d] > MEMD_STATIC_MAX_SITES) return MEMD_ERR_INVALID;
    if (__builtin_mul_overflow(V, (int64_t)mesh[d], &V)) return MEMD_ERR_INVALID;
  }
  if (V > MEMD_STATIC_MAX_SITES) return MEMD_ERR_INVALID;  // beyond the fixed scratch
  // an error left by the caller's earlier work is the caller's: refuse
  // without clearing it
  if (cudaPeekAtLastError() != cudaSuccess) return MEMD_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MEMD_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_static_partials) != cudaSuccess) {
        cudaGetLastError();
        return MEMD_ERR_CUDA;
      }
      g_addr[dev] = (double*)p;
    }
    scratch = g_addr[dev];
  }
  Mesh m{};
  for (int d = 0; d < 3; ++d) {
    m.n[d] = mesh[d];
    m.L[d] = mesh[d] * a;
  }
  m.V = V;
  m.a = a;
  const int nb = (int)((V + kSitesPerBlock - 1) / kSitesPerBlock);
  const double cB = dt / a, a3 = a * a * a;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)nb, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.stream = (cudaStream_t)cuda_stream;
  // each launch's own status: a failed launch is this call's error, cleared
  // here so that it does not surface in the caller's later work
  cudaError_t e =
      precision == MEMD_FP32
          ? cudaLaunchKernelEx(&cfg, k_energy_partials<float>, m, (const float*)D,
                               (const float*)B, (const float*)inv_eps, cB, scratch, nb)
          : cudaLaunchKernelEx(&cfg, k_energy_partials<double>, m, (const double*)D,
                               (const double*)B, (const double*)inv_eps, cB, scratch, nb);
  if (e == cudaSuccess) {
    cfg.gridDim = dim3(1, 1, 1);
    e = cudaLaunchKernelEx(&cfg, k_energy_finish, (const double*)scratch, nb, a3,
                           0.5 * c_light * c_light * a3, out2);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MEMD_ERR_CUDA;
  }
  return MEMD_OK;
}
