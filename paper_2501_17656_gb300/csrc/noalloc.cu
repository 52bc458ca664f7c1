// noalloc.cu -- h2mg_apply_noalloc: the H2 matrix-vector product with its scratch in
// a fixed device array instead of memory the library allocates.
//
// Some callers cannot call cudaMalloc at the point where they need a product: code
// inside an allocator callback (which must not re-enter the allocator), or processes
// whose device memory is entirely reserved up front by another allocator (a
// framework's caching pool), where a cudaMalloc would fail. This entry point allocates
// nothing: the product's workspace (coefficient buffers, point buffers and the row
// accumulators of the block products) lives in the file-scope array below, whose
// address is looked up once per device.
#include <mutex>
#include <string>

#include "internal.h"

namespace h2mg {

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[H2MG_NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[128] = {nullptr};

// Device address of the array on the current device (looked up on the first call
// made with that device current).
static unsigned char* scratch_address() {
  int dev = 0;
  H2_CUDA(cudaGetDevice(&dev));
  H2_REQUIRE(dev >= 0 && dev < 128, H2MG_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      throw Error{H2MG_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)};
    }
    g_noalloc_addr[dev] = p;
  }
  return (unsigned char*)g_noalloc_addr[dev];
}

static size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace h2mg

using namespace h2mg;

extern "C" h2mg_status h2mg_apply_noalloc(h2mg_matrix A, const double* x, double* y, void* stream) {
  try {
    set_error("");
    H2_REQUIRE(A && x && y, H2MG_ERR_INVALID_ARG, "null pointer argument");
    H2_REQUIRE(is_device_pointer(x) && is_device_pointer(y), H2MG_ERR_INVALID_ARG,
               "h2mg_apply_noalloc needs device vectors (host vectors would need staging memory)");
    Matrix& M = A->M;
    size_t coef, pts;
    apply_level1_ws_sizes(M, &coef, &pts);
    size_t need = 3 * up256(coef) + 2 * up256(pts);
    if (need > (size_t)H2MG_NOALLOC_SCRATCH_BYTES)
      throw Error{H2MG_ERR_UNSUPPORTED, "this matrix needs " + std::to_string(need) +
                                            " bytes of scratch; the fixed array holds " +
                                            std::to_string((size_t)H2MG_NOALLOC_SCRATCH_BYTES)};
    unsigned char* base = scratch_address();
    cudaStream_t s = (cudaStream_t)stream;
    ApplyWork ws;
    unsigned char* p = base;
    ws.xc = p; p += up256(coef);
    ws.yr = p; p += up256(coef);
    ws.yc = p; p += up256(coef);
    ws.xp = p; p += up256(pts);
    ws.yp = p;
    // The point buffer's padded slots must read as zero; the level-1 product clears
    // that buffer itself before filling it, so what an earlier call left in the array
    // does not leak into this one.
    bool prof = M.prof.on;
    M.prof.on = false;   // the event record could grow; keep this call allocation-free
    try {
      apply_level1_ws(M, x, y, s, ws);
    } catch (...) {
      M.prof.on = prof;
      throw;
    }
    M.prof.on = prof;
    return H2MG_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.status;
  } catch (...) {
    set_error("unknown error");
    return H2MG_ERR_CUDA;
  }
}
