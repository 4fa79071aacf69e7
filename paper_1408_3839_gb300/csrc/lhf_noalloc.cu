// lhf_noalloc.cu -- k-point eigensolve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside CUDA stream capture (allocation is
// not allowed there), services that must stay within a fixed device-memory budget set at
// start-up, and hosts whose allocator policy forbids raw CUDA allocations (another framework
// owns the memory).  For them lhf_k_point_eigensolve_noalloc runs the same kernels as
// lhf_k_point_eigensolve without a context: the descriptor and the kernels' scratch (the
// overlap norms s0 and a status word) live in one file-scope device array, sized once for all,
// that every GPU loading this library holds until the process exits.
#include <mutex>
#include <string.h>

#include "lhf_internal.cuh"

namespace {

constexpr size_t kScratchBytes = LHF_NOALLOC_SCRATCH_BYTES;
constexpr size_t kDescBytes = (sizeof(lhf::SysDev) + 255) / 256 * 256;
static_assert(kDescBytes + 256 + LHF_MAX_M0 * sizeof(double) <= kScratchBytes,
              "the no-alloc scratch must hold a descriptor, a status word and s0 for m0 = LHF_MAX_M0");

// Device scratch shared by every call on a device: [descriptor | status word | s0[m0]].
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_addr[kMaxDevices] = {};  // device address of g_scratch per device

// Device address of g_scratch on the current device (looked up once per device; the name
// g_scratch in host code is only a stand-in and must not be passed to a kernel).
cudaError_t scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[device];
  return cudaSuccess;
}

}  // namespace

extern "C" lhf_status lhf_k_point_eigensolve_noalloc(const int *L, int m0, const double *Hbar,
                                                     const double *Sbar, double *eig, int *k_status,
                                                     void *stream) {
  if (!L || !Hbar || !Sbar || !eig) return LHF_ERR_ARG;
  if (m0 < 1 || m0 > LHF_MAX_M0) return LHF_ERR_ARG;  // scratch holds s0 for m0 <= LHF_MAX_M0
  long long nblocks = 1;
  for (int l = 0; l < 3; ++l) {
    if (L[l] < 1 || L[l] > 4096) return LHF_ERR_ARG;
    nblocks *= L[l];
  }
  if (nblocks * m0 * m0 > (1ll << 31)) return LHF_ERR_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return LHF_ERR_CUDA;
  }
  unsigned char *base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return LHF_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  lhf::SysDev sd;
  memset(&sd, 0, sizeof sd);
  for (int l = 0; l < 3; ++l) sd.d[l].L = L[l];
  sd.m0 = m0;
  sd.nblocks = (int)nblocks;
  sd.box = 0;
  sd.Hbar = const_cast<double *>(Hbar);
  sd.Sbar = const_cast<double *>(Sbar);
  sd.eig = eig;
  sd.kstat = k_status;
  unsigned *flags = reinterpret_cast<unsigned *>(base + kDescBytes);
  sd.s0 = reinterpret_cast<double *>(base + kDescBytes + 256);
  lhf::SysDev *dsys = reinterpret_cast<lhf::SysDev *>(base);
  // sd is pageable host memory: the copy has been staged when cudaMemcpyAsync returns
  if (cudaMemcpyAsync(dsys, &sd, sizeof sd, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(flags, 0, sizeof(unsigned), st) != cudaSuccess ||
      lhf::launch_overlap_norms(dsys, 1, st) != cudaSuccess ||
      lhf::launch_eig(dsys, 1, (int)nblocks, m0, flags, nullptr, st, false) != cudaSuccess) {
    cudaGetLastError();
    return LHF_ERR_CUDA;
  }
  return LHF_OK;
}
