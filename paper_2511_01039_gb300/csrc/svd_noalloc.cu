// Scratch-free variant of the small FP64 SVD (fpeps_svd_f64): the same
// one-sided Jacobi kernels, with their working storage in a fixed device array
// instead of memory obtained from cudaMallocAsync.
//
// Who needs it: callers that must not allocate device memory at the moment
// they need the factorisation -- for example code running after a framework
// has reserved the whole device memory pool for its own allocator (so that
// cudaMallocAsync would fail or fight it), or a latency-critical loop in which
// an allocation could synchronise, fragment the pool or fail. They pass only
// their input and output buffers; this entry point allocates nothing.
//
// The working storage is g_svd_scratch below: 2 k^2 doubles (working matrix and
// accumulated rotations) + k ints (ordering) + 512 bytes of counters, for
// k <= FPEPS_SVD_NOALLOC_MAX_K (256), about 1.05 MB. Every GPU that loads the
// library holds it until the process exits. In host code the symbol names a
// host-side stand-in, not device memory, so it is never handed to a kernel
// directly: on the first call on a device (with that device current) its device
// address is looked up once with cudaGetSymbolAddress and cached; later calls
// on that device reuse it. The cached address belongs to the device's primary
// context: after cudaDeviceReset (which destroys that context) it is stale, so a
// process that resets a device must not call this entry point on it again. All
// calls share the array: calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it.
#include <exception>
#include <mutex>

#include "common.cuh"

namespace fpeps {
namespace {

constexpr int kMaxK = FPEPS_SVD_NOALLOC_MAX_K;
constexpr size_t kScratchBytes = 2 * (size_t)kMaxK * kMaxK * sizeof(double) + (size_t)kMaxK * sizeof(int) + 512;
static __device__ __align__(256) unsigned char g_svd_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {};

// device address of g_svd_scratch on the current device (looked up once per device)
char* scratch_address() {
  int dev = 0;
  FP_CUDA(cudaGetDevice(&dev));
  FP_CHECK(dev >= 0 && dev < 64, FPEPS_ERR_UNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    FP_CUDA(cudaGetSymbolAddress(&p, g_svd_scratch));
    FP_CHECK(p != nullptr, FPEPS_ERR_CUDA, "cudaGetSymbolAddress returned NULL");
    g_addr[dev] = p;
  }
  return static_cast<char*>(g_addr[dev]);
}

}  // namespace
}  // namespace fpeps

extern "C" fpeps_status fpeps_svd_f64_noalloc(const double* M, int32_t k, double* U, double* sigma, double* V,
                                              void* cuda_stream) {
  try {
    if (!M || !U || !sigma || !V || k < 1) throw fpeps::Error{FPEPS_ERR_ARG, "bad SVD arguments"};
    if (k > fpeps::kMaxK)
      throw fpeps::Error{FPEPS_ERR_ARG, "k exceeds FPEPS_SVD_NOALLOC_MAX_K (256): use fpeps_svd_f64"};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    char* scr = fpeps::scratch_address();
    const size_t kk = (size_t)k * k;
    double* Mw = reinterpret_cast<double*>(scr);
    double* Vw = Mw + kk;
    int* order = reinterpret_cast<int*>(Vw + kk);
    char* ws = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(order + k) + 255) & ~uintptr_t(255));
    int* info = reinterpret_cast<int*>(ws + 128);
    // every region is rewritten before it is read: Mw by this copy, Vw, order and
    // the counters by the Jacobi kernels (which reset their counters on entry)
    FP_CUDA(cudaMemcpyAsync(Mw, M, kk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    fpeps::svd_jacobi_f64(s, Mw, k, U, sigma, Vw, order, info, ws);
    fpeps::gather_cols_f64(s, Vw, order, k, V);
    FP_CUDA(cudaStreamSynchronize(s));
    return FPEPS_OK;
  } catch (const fpeps::Error& e) {
    return e.st;
  } catch (const std::exception&) {
    return FPEPS_ERR_ARG;
  }
}
