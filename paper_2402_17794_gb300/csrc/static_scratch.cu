// Y = A X in FP64 without a plan and without any device allocation.
//
// Who needs this: code that runs where it may not call cudaMalloc -- e.g. a
// callback or plugin embedded in a host framework that owns all device
// memory and forbids allocation inside the call, a stream-ordered section
// whose caller has handed over only its inputs and outputs, or a process that
// has already reserved the whole device.  Such callers cannot size or own a
// plan workspace, so this entry point keeps its split-K partial sums in one
// fixed array compiled into the library instead.
//
// The array lives for as long as the library is loaded, on every GPU that
// loads it, and is shared by every call: calls that overlap on the GPU (two
// streams, or two host threads) race on it.  Nothing in it needs to start at
// zero: every partial slice a call reads back is written whole by that same
// call first.  Its device address is looked up with cudaGetSymbolAddress the
// first time a device uses the entry point (with that device current); that
// first call therefore makes a runtime query and should happen before any
// stream capture that includes this entry point.
#include <mutex>

#include "internal.h"

namespace rsvd {
namespace {

// 4 Mi doubles = 32 MiB of split-K partials.
constexpr size_t kStaticScratchDoubles = (size_t)4 << 20;
static __device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

// Resolves (once per device) the scratch's device address and the SM count.
int device_setup(double** scratch, int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RSVD_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RSVD_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return RSVD_ERR_CUDA;
    g_scratch_ptr[dev] = (double*)p;
    g_num_sms[dev] = sms;
  }
  *scratch = g_scratch_ptr[dev];
  *num_sms = g_num_sms[dev];
  return RSVD_OK;
}

}  // namespace
}  // namespace rsvd

extern "C" int rsvd_apply_a_f64_static(const double* A, int64_t m, int64_t n, int64_t lda,
                                       const double* X, int64_t ldx, int l, double* Y,
                                       int64_t ldy, void* cuda_stream) {
  using namespace rsvd;
  if (!A) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (lda < m) return -4;
  if (!X) return -5;
  if (ldx < n) return -6;
  if (l < 1) return -7;
  if (!Y) return -8;
  if (ldy < m) return -9;
  // at least one m x l partial slice must fit the fixed scratch
  if ((size_t)m * (size_t)l > kStaticScratchDoubles) return RSVD_ERR_WORKSPACE;
  double* scratch = nullptr;
  int sms = 0;
  int rc = device_setup(&scratch, &sms);
  if (rc) return rc;
  GemmArgs<double> g{A, lda, false, X, ldx, Y, ldy, m, n, l};
  if (launch_gemm<double>(g, scratch, kStaticScratchDoubles, sms, (cudaStream_t)cuda_stream) !=
      cudaSuccess)
    return RSVD_ERR_CUDA;
  return RSVD_OK;
}
