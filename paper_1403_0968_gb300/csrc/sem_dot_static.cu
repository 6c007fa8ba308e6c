// Allocation-free FP64 inner product: the sem_dot reduction with its scratch in a fixed
// file-scope device array instead of a caller-allocated workspace.
//
// Who needs it: code that must not allocate device memory at the point where it needs a dot
// product — for example a solver step running inside a host framework that owns all device
// memory through its own pool, or a real-time loop that forbids cudaMalloc after start-up
// (cudaMalloc may synchronise the device and can fail under memory pressure).  Such a caller
// passes only its input vectors and a device pointer for the result.
//
// Scratch: SEM_DOT_STATIC_BLOCKS FP64 partial sums plus one ticket counter, held in a static
// __device__ array for as long as the library is loaded (about 8 KB on every GPU that loads it).
// In host code the array's name is only a host-side stand-in, so its device address is fetched
// with cudaGetSymbolAddress once per device, on the first call made while that device is current
// (that call also clears the ticket counter and synchronises the device, so make it before any
// stream capture).  Every call shares the one array: calls whose kernels overlap on the GPU (two
// streams, or two host threads) race on it and must be serialised by the caller.  The address is
// cached per device for the life of the process: after cudaDeviceReset the module is loaded again
// in a new context and the cached address is stale, so the function is not for use across a reset.
#include <mutex>

#include "sem_internal.h"
#include "sem_reduce.cuh"

#define SEM_DOT_STATIC_BLOCKS 1024
#define SEM_DOT_STATIC_THREADS 256
#define SEM_DOT_STATIC_MAX_DEVICES 128
// each thread walks at most 4096 grid-stride steps: n <= 1024 * 256 * 4096 = 2^30
#define SEM_DOT_STATIC_MAX_N ((int64_t)SEM_DOT_STATIC_BLOCKS * SEM_DOT_STATIC_THREADS * 4096)

// [0, BLOCKS): per-block partial sums; slot BLOCKS: the ticket counter (as unsigned int)
static __device__ __align__(256) double g_dot_scratch[SEM_DOT_STATIC_BLOCKS + 32];

namespace {
std::mutex g_mu;
double *g_scratch[SEM_DOT_STATIC_MAX_DEVICES];

__global__ void __launch_bounds__(SEM_DOT_STATIC_THREADS)
    k_dot_static(int64_t n, const double *x, const double *y, double *out, double *scratch) {
  constexpr int NT = SEM_DOT_STATIC_THREADS;
  __shared__ double s_red[32];
  __shared__ int s_flag;
  unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + SEM_DOT_STATIC_BLOCKS);
  double acc = 0.0;
  for (int64_t g = (int64_t)blockIdx.x * NT + threadIdx.x; g < n; g += (int64_t)gridDim.x * NT) acc += x[g] * y[g];
  const double bs = block_sum<NT>(acc, s_red);
  if (publish_partial<NT>(bs, scratch, ticket, s_red, &s_flag)) {
    const double tot = final_sum<NT>(scratch, gridDim.x, s_red);
    if (threadIdx.x == 0) {
      *out = tot;
      *ticket = 0;  // leave the counter cleared for the next call
    }
  }
}

// Device address of the scratch array on the current device (set-up on first use).
sem_status scratch_for_current_device(double **out) {
  int dev = 0;
  SEM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= SEM_DOT_STATIC_MAX_DEVICES) return sem_fail(SEM_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    // the ticket must start at zero
    e = cudaMemset(static_cast<double *>(p) + SEM_DOT_STATIC_BLOCKS, 0, 32 * sizeof(double));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return sem_fail(SEM_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));
    g_scratch[dev] = static_cast<double *>(p);
  }
  *out = g_scratch[dev];
  return SEM_OK;
}
}  // namespace

extern "C" sem_status sem_dot_static(int64_t n, const double *d_x, const double *d_y, double *d_out,
                                     sem_stream_t stream) {
  if (n < 0 || n > SEM_DOT_STATIC_MAX_N)
    return sem_fail(SEM_ERR_INVALID, "sem_dot_static: n must be in [0, 2^30] (size of the static scratch)");
  if (!d_out || (n > 0 && (!d_x || !d_y))) return sem_fail(SEM_ERR_INVALID, "NULL argument");
  double *scratch = nullptr;
  sem_status st = scratch_for_current_device(&scratch);
  if (st != SEM_OK) return st;
  int64_t blocks = (n + SEM_DOT_STATIC_THREADS - 1) / SEM_DOT_STATIC_THREADS;
  if (blocks < 1) blocks = 1;
  if (blocks > SEM_DOT_STATIC_BLOCKS) blocks = SEM_DOT_STATIC_BLOCKS;
  k_dot_static<<<(unsigned)blocks, SEM_DOT_STATIC_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, d_x, d_y, d_out, scratch);
  SEM_CUDA_TRY(cudaGetLastError());
  return SEM_OK;
}
