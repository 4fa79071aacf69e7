// lhf_noalloc.cu -- k-point eigensolve for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: services that must stay within a fixed device-memory
// budget set at start-up (an allocation later could fail or evict another tenant's memory), and
// hosts whose allocator policy forbids raw CUDA allocations because another framework owns the
// device memory.  For them lhf_k_point_eigensolve_noalloc runs the same kernels as
// lhf_k_point_eigensolve without a context: the descriptor and the kernels' scratch (the
// overlap norms s0 and a status word) live in one file-scope device array, sized once for all,
// that every GPU loading this library holds until the process exits.  The descriptor is written
// into that array by a one-thread-block kernel that receives its fields as kernel arguments, so
// no host buffer has to outlive the call.
#include <mutex>

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

// The fields of the descriptor that the overlap-norm and k-point kernels read for one system.
struct NoallocArgs {
  int L[3];
  int m0;
  int nblocks;
  const double *Hbar, *Sbar;
  double *eig;
  int *kstat;
};

// Writes the descriptor [0, kDescBytes) and the status word of the scratch at base: every byte of
// the descriptor zero except the fields above, s0 pointing into the scratch.
__global__ void k_noalloc_setup(NoallocArgs a, unsigned char *base) {
  unsigned *words = reinterpret_cast<unsigned *>(base);
  for (size_t i = threadIdx.x; i < kDescBytes / sizeof(unsigned); i += blockDim.x) words[i] = 0u;
  if (threadIdx.x == 0) *reinterpret_cast<unsigned *>(base + kDescBytes) = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    lhf::SysDev *sd = reinterpret_cast<lhf::SysDev *>(base);
    for (int l = 0; l < 3; ++l) sd->d[l].L = a.L[l];
    sd->m0 = a.m0;
    sd->nblocks = a.nblocks;
    sd->box = 0;
    sd->Hbar = const_cast<double *>(a.Hbar);
    sd->Sbar = const_cast<double *>(a.Sbar);
    sd->eig = a.eig;
    sd->kstat = a.kstat;
    sd->s0 = reinterpret_cast<double *>(base + kDescBytes + 256);
  }
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
  NoallocArgs a;
  for (int l = 0; l < 3; ++l) a.L[l] = L[l];
  a.m0 = m0;
  a.nblocks = (int)nblocks;
  a.Hbar = Hbar;
  a.Sbar = Sbar;
  a.eig = eig;
  a.kstat = k_status;
  unsigned *flags = reinterpret_cast<unsigned *>(base + kDescBytes);
  lhf::SysDev *dsys = reinterpret_cast<lhf::SysDev *>(base);
  k_noalloc_setup<<<1, 256, 0, st>>>(a, base);
  if (cudaGetLastError() != cudaSuccess ||
      lhf::launch_overlap_norms(dsys, 1, st) != cudaSuccess ||
      lhf::launch_eig(dsys, 1, (int)nblocks, m0, flags, nullptr, st, false) != cudaSuccess) {
    cudaGetLastError();
    return LHF_ERR_CUDA;
  }
  return LHF_OK;
}
