// noalloc.cu -- mdbs_field_stats_static: the field-statistics reduction
// (liquid volume, alpha min / max, non-finite sentinel) for callers that
// cannot allocate device memory.  Its scratch (per-block partial results)
// lives in a file-scope __device__ array instead of a cudaMalloc'ed arena.
#include <math.h>

#include <mutex>

#include "../../include/mdbs.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 4 channels (volume, min, max, non-finite count) x MDBS_STATIC_STATS_MAX_BLOCKS partials.
// Every device that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_stats_scratch[4 * MDBS_STATIC_STATS_MAX_BLOCKS];

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};  // device address of g_stats_scratch, per device

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// stage 1: each block writes its partials into the static scratch
__global__ void k_stats_partials(long long cells, double volume, const double* __restrict__ phi,
                                 const double* __restrict__ alpha, const double* __restrict__ p,
                                 double* __restrict__ scratch, int nb) {
  double mass = 0.0, amin = INFINITY, amax = -INFINITY, bad = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x) {
    const double a = alpha[c];
    mass += phi[c] * a * volume;
    amin = fmin(amin, a);
    amax = fmax(amax, a);
    if (!isfinite(a) || !isfinite(p[c])) bad += 1.0;
  }
  __shared__ double sm[4][kThreads / 32];
  mass = warp_sum(mass);
  bad = warp_sum(bad);
  amin = warp_min(amin);
  amax = warp_max(amax);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sm[0][w] = mass;
    sm[1][w] = amin;
    sm[2][w] = amax;
    sm[3][w] = bad;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = INFINITY, s2 = -INFINITY, s3 = 0.0;
    for (int i = 0; i < kThreads / 32; i++) {
      s0 += sm[0][i];
      s1 = fmin(s1, sm[1][i]);
      s2 = fmax(s2, sm[2][i]);
      s3 += sm[3][i];
    }
    scratch[blockIdx.x] = s0;
    scratch[nb + blockIdx.x] = s1;
    scratch[2 * nb + blockIdx.x] = s2;
    scratch[3 * nb + blockIdx.x] = s3;
  }
}

// stage 2: one thread folds the partials in a fixed order into the caller's output
__global__ void k_stats_final(const double* __restrict__ scratch, int nb, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double mass = 0.0, amin = INFINITY, amax = -INFINITY, bad = 0.0;
  for (int b = 0; b < nb; b++) {
    mass += scratch[b];
    amin = fmin(amin, scratch[nb + b]);
    amax = fmax(amax, scratch[2 * nb + b]);
    bad += scratch[3 * nb + b];
  }
  out[0] = mass;
  out[1] = amin;
  out[2] = amax;
  out[3] = bad;
}

// Device address of the static scratch on the current device, looked up once per
// device (cudaGetSymbolAddress) with that device current.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_stats_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (double*)ptr;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int mdbs_field_stats_static(int64_t cells, double cell_volume, const double* porosity,
                                       const double* alpha, const double* p, double* out, void* stream) {
  if (cells < 1 || cells > MDBS_STATIC_STATS_MAX_CELLS) return MDBS_ERR_ARG;
  if (!porosity || !alpha || !p || !out || !(cell_volume > 0.0)) return MDBS_ERR_ARG;
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return MDBS_ERR_CUDA;
  long long blocks = (cells + kThreads - 1) / kThreads;
  const int nb = (int)(blocks < MDBS_STATIC_STATS_MAX_BLOCKS ? blocks : MDBS_STATIC_STATS_MAX_BLOCKS);
  cudaStream_t s = (cudaStream_t)stream;
  // An error already pending on this thread belongs to the caller's earlier work: report
  // it as MDBS_ERR_CUDA without launching and leave it pending (cudaPeekAtLastError does
  // not clear it).  Otherwise any error after the launches is theirs and is cleared.
  if (cudaPeekAtLastError() != cudaSuccess) return MDBS_ERR_CUDA;
  k_stats_partials<<<nb, kThreads, 0, s>>>(cells, cell_volume, porosity, alpha, p, scratch, nb);
  k_stats_final<<<1, 32, 0, s>>>(scratch, nb, out);
  return cudaGetLastError() == cudaSuccess ? MDBS_OK : MDBS_ERR_CUDA;
}
