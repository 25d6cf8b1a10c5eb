// runtime.cu -- host-side services shared by the entry points:
//   - the device error word: kernels whose bounded waits run out OR a site
//     bit into one word of page-locked, device-mapped host memory, which the
//     host reads without synchronising the device (omerf_sync and the next
//     call of the affected entry point report it as OMERF_ETIMEOUT);
//   - host fault injection for tests: OMERF_FAULT names sites that then fail
//     as if the CUDA call there had failed, without touching the GPU, or (for
//     a device wait) that make the wait give up at once;
//   - NVTX ranges around every entry point, visible to profilers.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace omerf {

bool fault_injected(const char* site) {
  const char* v = std::getenv("OMERF_FAULT");
  if (!v || !*v) return false;
  const size_t n = std::strlen(site);
  for (const char* p = v;;) {
    const char* e = std::strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : std::strlen(p);
    if (len == n && std::strncmp(p, site, n) == 0) return true;
    if (!e) return false;
    p = e + 1;
  }
}

omerf_status injected_launch_failure(const char* entry) {
  set_error("%s: launch failed (fault injected by OMERF_FAULT=launch)", entry);
  return OMERF_ECUDA;
}

static std::atomic<unsigned*> g_err_host{nullptr};
static unsigned* g_err_dev = nullptr;
static std::once_flag g_err_once;

unsigned* device_error_word() {
  std::call_once(g_err_once, [] {
    void* h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    std::memset(h, 0, 64);
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess || !d) {
      cudaGetLastError();
      cudaFreeHost(h);
      return;
    }
    g_err_dev = static_cast<unsigned*>(d);
    g_err_host.store(static_cast<unsigned*>(h), std::memory_order_release);
  });
  return g_err_host.load(std::memory_order_acquire) ? g_err_dev : nullptr;
}

omerf_status take_device_error() {
  unsigned* h = g_err_host.load(std::memory_order_acquire);
  if (!h) return OMERF_OK;
  const unsigned v = __atomic_exchange_n(h, 0u, __ATOMIC_SEQ_CST);
  if (!v) return OMERF_OK;
  set_error("a bounded device-side wait gave up:%s%s%s; the output of that call is incomplete",
            (v & kErrExtractWait) ? " brick extraction waited too long for a tensor copy" : "",
            (v & kErrExtractDrain) ? " (and for the copy still in flight)" : "",
            (v & kErrMlpWait) ? " the MLP backward waited too long for a tensor-core product" : "");
  return OMERF_ETIMEOUT;
}

ApiRange::ApiRange(const char* name) { nvtxRangePushA(name); }
ApiRange::~ApiRange() { nvtxRangePop(); }

}  // namespace omerf
