// Allocation-free variant of tt_dot for callers that cannot allocate device
// memory (see tt_dot_noalloc in include/ttsg.h).
//
// The Gram sweep's scratch lives in the file-scope device array below, which
// every GPU that loads this library holds until the process exits.  In host
// code the array's name is only a host-side stand-in, so its device address is
// looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached; that look-up happens in the first call on each device.
#include "common.cuh"
#include <mutex>

namespace ttsg {
size_t dot_bytes_without_splitk(int mode, const tt_vec* x, const tt_vec* y, int* code);
int dot_on_workspace_without_splitk(int mode, const tt_vec* x, const tt_vec* y, double* out,
                                    void* ws, size_t bytes, void* stream);
}  // namespace ttsg

static __device__ __align__(256) unsigned char tt_noalloc_scratch[TT_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[TT_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up on first use).
int noalloc_scratch(void** ptr) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    ttsg::set_last_error(std::string("tt_dot_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return TT_ERR_CUDA;
  }
  if (dev < 0 || dev >= TT_MAX_DEVICES) {
    ttsg::set_last_error("tt_dot_noalloc: device index beyond TT_MAX_DEVICES");
    return TT_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, tt_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      ttsg::set_last_error(std::string("tt_dot_noalloc: cudaGetSymbolAddress: ") +
                           cudaGetErrorString(e));
      return TT_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *ptr = g_noalloc_ptr[dev];
  return TT_OK;
}
}  // namespace

int tt_dot_noalloc(int mode, const tt_vec* x, const tt_vec* y, double* out, void* stream) {
  // size check on the host before touching the device
  int code = TT_OK;
  const size_t need = ttsg::dot_bytes_without_splitk(mode, x, y, &code);
  if (need == 0) return code;  // the query's own status; message already set
  if (need > (size_t)TT_NOALLOC_SCRATCH_BYTES) {
    ttsg::set_last_error("tt_dot_noalloc: these ranks need " + std::to_string(need) +
                         " bytes of scratch, more than the fixed " +
                         std::to_string((size_t)TT_NOALLOC_SCRATCH_BYTES) +
                         " bytes; use tt_dot with a workspace");
    return TT_ERR_ARG;
  }
  void* ws = nullptr;
  const int rc = noalloc_scratch(&ws);
  if (rc != TT_OK) return rc;
  return ttsg::dot_on_workspace_without_splitk(mode, x, y, out, ws, TT_NOALLOC_SCRATCH_BYTES,
                                               stream);
}
