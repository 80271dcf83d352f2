// sbfwi_misfit_noalloc: the misfit reduction without any device allocation.
//
// sbfwi_misfit stages its per-block partial sums in a buffer it allocates with
// cudaMalloc on every call.  Some callers cannot let a library allocate device
// memory: a host framework that has reserved (nearly) all of HBM in its own
// caching pool, a real-time loop that must not hit the driver's allocator or
// its implicit synchronisation, or a process running under a fixed memory
// budget.  This entry point keeps its partial sums in a fixed, file-scope device
// array instead, so a call touches only the caller's buffers and that array.
//
// The array is a module-level __device__ variable: every device that loads the
// library holds it (32 KiB) until the process exits.  Its address is looked up
// with cudaGetSymbolAddress once per device, on the first call made with that
// device current; make that first call before capturing the stream into a CUDA
// graph.  All calls share the array: two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it and may return wrong
// values.  Each block overwrites its own partial sum, so nothing is carried over
// from an earlier call.
#include <mutex>
#include <string>

#include "internal.h"
#include "prof.h"

namespace sbfwi {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunk = 65536;        // trace samples reduced by one block
constexpr int kMaxParts = 4096;          // blocks, so n <= kMaxParts * kChunk
constexpr int kMaxDevices = 64;

// per-block partial sums of (observed - traces)^2
static __device__ __align__(256) double g_noalloc_partials[kMaxParts];

std::mutex g_mu;
double* g_partials_addr[kMaxDevices] = {};

__global__ void noalloc_partial_kernel(const double* tr, const double* ob, int64_t n, double* res, double* partial) {
  __shared__ double red[kThreads];
  const int64_t lo = (int64_t)blockIdx.x * kChunk;
  const int64_t hi = lo + kChunk < n ? lo + kChunk : n;
  double acc = 0.0;
  for (int64_t t = lo + threadIdx.x; t < hi; t += kThreads) {
    const double d = ob[t] - tr[t];
    if (res) res[t] = d;
    acc = fma(d, d, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void noalloc_final_kernel(const double* partial, int parts, double half_dt, double* E) {
  __shared__ double red[kThreads];
  double acc = 0.0;
  for (int t = threadIdx.x; t < parts; t += kThreads) acc += partial[t];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) E[0] = half_dt * red[0];
}

bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace sbfwi

using namespace sbfwi;

extern "C" int sbfwi_misfit_noalloc(const double* traces, const double* observed, int64_t n, double dt, double* E_out,
                                    double* residual_out, void* stream) {
  if (!traces || !observed || !E_out) return fail(SBFWI_EINVAL, "NULL argument");
  if (n < 0) return fail(SBFWI_EINVAL, "n < 0");
  if (n > (int64_t)kMaxParts * kChunk)
    return fail(SBFWI_EINVAL, "n = " + std::to_string(n) + " exceeds the no-allocation limit of " +
                                  std::to_string((int64_t)kMaxParts * kChunk) + " trace samples");
  if (!on_device(traces) || !on_device(observed) || !on_device(E_out) || (residual_out && !on_device(residual_out)))
    return fail(SBFWI_EINVAL, "sbfwi_misfit_noalloc takes device pointers only");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(SBFWI_EUNSUPPORTED, "device index too large");
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_addr[dev]) {
      // the host-side name of the array is only a stand-in: its device address must be asked for
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&g_partials_addr[dev]), g_noalloc_partials);
      if (e != cudaSuccess) {
        g_partials_addr[dev] = nullptr;
        return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partials)");
      }
    }
    partials = g_partials_addr[dev];
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int parts = (int)((n + kChunk - 1) / kChunk);
  if (parts > 0) noalloc_partial_kernel<<<parts, kThreads, 0, st>>>(traces, observed, n, residual_out, partials);
  noalloc_final_kernel<<<1, kThreads, 0, st>>>(partials, parts, 0.5 * dt, E_out);
  profiler().count(kPhaseOther, parts > 0 ? 2 : 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "misfit kernels");
  return SBFWI_OK;
}
