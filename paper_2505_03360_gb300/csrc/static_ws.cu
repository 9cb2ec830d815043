// coll_eval_batch_static: the collision evaluation for callers that cannot
// allocate device memory.  The kernel's scratch lives in one file-scope device
// array of fixed size instead of a caller-provided workspace.
//
// Host code cannot use the array's name as a device address (on the host it
// names a shadow variable), so the address is looked up once per device with
// cudaGetSymbolAddress, the first time the entry point runs with that device
// current, and cached.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "coll_internal.h"
#include "../../include/coll.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB per device, held until exit
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::atomic<bool> g_scratch_ready[kMaxDevices];

// Address of the array on the current device (set-up on first use).
cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (g_scratch_ready[dev].load(std::memory_order_acquire)) {
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ready[dev].load(std::memory_order_relaxed)) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      (void)cudaGetLastError();   // not left behind for the next launch check to report
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    g_scratch_ptr[dev] = p;
    g_scratch_ready[dev].store(true, std::memory_order_release);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" coll_status coll_eval_batch_static(coll_plan p, const void* f, void* Q, int64_t n_cells,
                                              coll_stream stream) {
  if (!p || n_cells < 0) return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !Q || f == Q) return COLL_EINVAL;
  if (p->galerkin) return COLL_EUNSUPPORTED;    // the Galerkin mode's padded buffers scale with the batch
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return COLL_EINVAL;
  const int v = p->variant;
  const size_t per_cta = p->lay[v].ws_bytes_per_cta();
  const long long C = p->lay[v].cluster > 0 ? p->lay[v].cluster : 1;   // CTAs per cell
  long long grid = static_cast<long long>(p->num_sms) * p->ctas_per_sm[v];
  if (grid > n_cells * C) grid = n_cells * C;
  if (per_cta > 0) {
    const long long fit = static_cast<long long>(kStaticScratchBytes / per_cta);
    if (fit < C) return COLL_ENOMEM;            // one cell's scratch exceeds the fixed array
    if (grid > fit) grid = fit;                  // fewer resident CTAs, each loops over more cells
  }
  grid = grid / C * C;                           // whole clusters
  void* ws = nullptr;
  if (scratch_address(dev, &ws) != cudaSuccess) return COLL_ECUDA;
  coll::CollArgs a;
  a.f = f;
  a.Q = Q;
  a.n_cells = n_cells;
  a.tab = p->tab_dev;
  a.n_terms = p->n_terms;
  a.ws = ws;
  a.ws_per_cta = per_cta;
  a.status = p->status_dev;
  const int e = coll::launch_collision(p->Nk, p->ctype, p->io_f64, v, a, int(grid), stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}
