// lpa_noalloc.cu -- modularity without any device allocation.
//
// Some callers cannot allocate device memory at the moment they want a result: a host
// application whose own caching allocator already holds nearly all of the GPU's memory
// (so a cudaMalloc would fail or fragment its pool), or a latency-critical loop where a
// cudaMalloc / cudaFree would stall the device.  lpa_modularity_noalloc serves them: its
// scratch is the file-scope device array below, reserved once when the library's module
// is loaded on a GPU and held until the process exits.  The caller passes only the
// graph, the labels and the result pointer.
#include <cstdio>
#include <mutex>

#include "../../include/lpa.h"
#include "lpa_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kMaxPartials = 4096;  // per-block partial triples of the modularity kernels
// Sigma_c for up to LPA_NOALLOC_MAX_N labels, then partials, four results, an error word.
constexpr size_t kScratchDoubles = (size_t)LPA_NOALLOC_MAX_N + 3 * kMaxPartials + 4 + 4;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per device.
int scratch_on_current_device(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lpa::set_last_error(LPA_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return lpa::set_last_error(LPA_EUNSUPPORTED, "device ordinal too large for the static scratch table");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return lpa::set_last_error(LPA_ECUDA, cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_addr[dev]);
  return LPA_OK;
}

}  // namespace

extern "C" lpa_status lpa_modularity_noalloc(const int64_t* offsets, const int32_t* indices,
                                             const float* weights, int32_t n, int64_t m,
                                             const int32_t* labels, double* q_out,
                                             const lpa_options* opt) {
  char msg[256];
  const int chk = lpa::check_modularity_args(offsets, indices, n, m, labels, q_out);
  if (chk != LPA_OK) return (lpa_status)chk;
  if (n > LPA_NOALLOC_MAX_N) {
    snprintf(msg, sizeof(msg), "n = %d exceeds the static scratch limit of %d vertices", n,
             LPA_NOALLOC_MAX_N);
    return (lpa_status)lpa::set_last_error(LPA_EINVAL, msg);
  }
  const int npart = lpa::modularity_partials(n);
  if ((size_t)npart > kMaxPartials)
    return (lpa_status)lpa::set_last_error(LPA_EINTERNAL, "partials exceed the static scratch");
  double* scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st != LPA_OK) return (lpa_status)st;
  double* sigma_c = scratch;
  double* partials = scratch + LPA_NOALLOC_MAX_N;
  double* out4 = partials + 3 * kMaxPartials;
  int32_t* err = reinterpret_cast<int32_t*>(out4 + 4);
  cudaStream_t s = opt ? (cudaStream_t)opt->stream : nullptr;
  const bool validate = opt ? (opt->flags & LPA_VALIDATE) != 0 : true;
  cudaError_t e = cudaSuccess;
  if (validate) {
    int32_t host_err = 0;
    e = lpa::launch_fill_i32(err, 0, 1, s);
    if (e == cudaSuccess) e = lpa::launch_validate(offsets, indices, weights, n, m, labels, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return (lpa_status)lpa::set_last_error(LPA_ECUDA, cudaGetErrorString(e));
    if (host_err) {
      snprintf(msg, sizeof(msg), "invalid input (error bits 0x%x)", host_err);
      return (lpa_status)lpa::set_last_error(LPA_EINVAL, msg);
    }
  }
  // launch_modularity clears Sigma_c before accumulating and writes every partial it
  // reads, so the contents left by an earlier call do not matter
  double host_out[4] = {0, 0, 0, 0};
  e = lpa::launch_modularity(offsets, indices, weights, m, labels, n, sigma_c, partials, npart, out4, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, out4, sizeof(host_out), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return (lpa_status)lpa::set_last_error(LPA_ECUDA, cudaGetErrorString(e));
  *q_out = host_out[3];
  return LPA_OK;
}
