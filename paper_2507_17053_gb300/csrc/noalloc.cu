// FP64 continuous Galerkin apply that allocates nothing, for callers that
// cannot call cudaMalloc at the point where they apply the operator: code
// running while a CUDA graph is being captured into a memory pool they do
// not own, real-time loops whose allocator is locked after start-up, or
// host frameworks that hand the library only fixed buffers.
//
// The apply's scratch -- the per-face results of the surrogate-face kernel
// and the per-colour accumulation buffers of the cell kernel -- lives in one
// file-scope device array of kStaticScratchBytes (64 MiB).  The CUDA runtime
// reserves it on every GPU that loads this library, for the life of the
// process.  Host code cannot use the array's name as a device address, so
// the address is looked up once per device with cudaGetSymbolAddress (the
// first call on a device does this, with that device current) and cached.
#include <mutex>

#include "internal.hpp"

namespace sbm {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_scratch_mu;
static void* g_scratch_addr[kMaxDevices] = {};

static size_t round_up_256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace sbm

using namespace sbm;

extern "C" int sbm_apply_f64_noalloc(sbm_problem* prob, const double* x, double* y, void* stream) {
  if (!prob || !x || !y || x == y) return sbm_fail_detail(SBM_ERR_ARG, "bad vector argument");
  if (!prob->on_device) return sbm_fail_detail(SBM_ERR_STATE, "sbm_setup_face_data not called");
  if (prob->hp.desc.dg)
    return sbm_fail_detail(SBM_ERR_UNSUPPORTED, "sbm_apply_f64_noalloc serves CG problems only");
  const DeviceData& dd = prob->dd;
  const size_t face_bytes = round_up_256((size_t)dd.nface * 2 * prob->hp.L * sizeof(double));
  const size_t colour_bytes = (size_t)dd.ncolours * (size_t)prob->hp.n_dofs * sizeof(double);
  if (face_bytes + colour_bytes > kStaticScratchBytes)
    return sbm_fail_detail(SBM_ERR_ARG,
                           "problem needs " + std::to_string(face_bytes + colour_bytes) +
                               " bytes of scratch; the static buffer holds " +
                               std::to_string(kStaticScratchBytes));
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetDevice");
  if (dev != prob->device)
    return sbm_fail_detail(SBM_ERR_STATE, "current device is not the problem's device");
  if (dev < 0 || dev >= kMaxDevices) return sbm_fail_detail(SBM_ERR_ARG, "device index too large");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "cudaGetSymbolAddress");
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  // Every element of both regions that a kernel reads is written earlier in
  // the same call (all faces' results; colour buffers only where the DoF's
  // colour mask is set), so nothing has to be cleared first.
  double* face_scratch = reinterpret_cast<double*>(base);
  double* colour_scratch = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + face_bytes);
  // the same cell tile shape as sbm_apply_f64 (the autotuned or pinned one)
  e = launch_cg_apply_scratch<double>(prob->hp, dd, x, y, face_scratch, colour_scratch,
                                      dd.variant[0], (cudaStream_t)stream);
  if (e != cudaSuccess) return sbm_cuda_fail_detail(e, "sbm_apply_f64_noalloc");
  return SBM_OK;
}
