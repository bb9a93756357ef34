// Morton-key sort of particle positions with all scratch memory in one
// file-scope device array: for callers that cannot allocate device memory.
#include <mutex>

#include "hpm_internal.cuh"

namespace hpm {
namespace {

constexpr int64_t kMaxN = HPM_STATIC_SORT_MAX_N;
// the sort's histogram and offsets (2 x digits x sort tiles ints) and the
// status words of the scan over the histogram, sized from the sort's own
// constants so that radix_sort_pairs never finds its scratch too small
constexpr int64_t kHistInts = sort_scratch_ints(kMaxN);
constexpr int64_t kScanStatus = scan_tiles_of(kHistInts / 2) + 64;
constexpr size_t kHeader = 256;                              // error word
constexpr size_t kKeysOff = kHeader;
constexpr size_t kPermOff = kKeysOff + sizeof(uint64_t) * kMaxN;
constexpr size_t kHistOff = kPermOff + sizeof(uint32_t) * kMaxN;
constexpr size_t kHistBytes = sizeof(int) * kHistInts;
static_assert(kHistBytes >= sizeof(int) * sort_scratch_ints(kMaxN), "histogram scratch");
static_assert(kScanStatus >= scan_tiles_of(kHistInts / 2), "scan status words");
constexpr size_t kScanOff = (kHistOff + kHistBytes + 255) / 256 * 256;  // ticket, then status words
constexpr size_t kBytes = kScanOff + 256 + sizeof(unsigned long long) * kScanStatus;

// Held by every device that loads the library, for the life of the process.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the symbol itself as a device address).
hpm_status scratch_address(void **out) {
  int dev = 0;
  HPM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return HPM_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    HPM_CUDA(cudaGetSymbolAddress(&p, g_sort_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HPM_OK;
}

}  // namespace
}  // namespace hpm

using namespace hpm;

extern "C" hpm_status hpm_sort_particles_static(const hpm_domain *dom, int max_depth, const double *d_pos,
                                                int64_t n, uint64_t *d_keys, uint32_t *d_perm, void *stream) {
  if (!dom || max_depth < 0 || max_depth > kMaxDepth || n < 0) return HPM_ERR_INVALID_ARG;
  if (n > kMaxN) return HPM_ERR_INVALID_ARG;  // beyond the static scratch
  if (!(dom->side > 0.0)) return HPM_ERR_INVALID_ARG;
  if (n == 0) return HPM_OK;
  if (!d_pos || !d_keys || !d_perm) return HPM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  void *base = nullptr;
  HPM_TRY(scratch_address(&base));
  unsigned char *b = static_cast<unsigned char *>(base);
  int *err = reinterpret_cast<int *>(b);
  HPM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  HPM_TRY(launch_morton_keys(*dom, max_depth, d_pos, n, d_keys, err, st));
  // views into the static array: ensure() finds them large enough and allocates nothing
  DevBuf hist;
  hist.p = b + kHistOff;
  hist.cap = kHistBytes;
  uint64_t *k0 = d_keys, *k1 = reinterpret_cast<uint64_t *>(b + kKeysOff);
  uint32_t *v0 = d_perm, *v1 = reinterpret_cast<uint32_t *>(b + kPermOff);
  // the scan's control words (zero when the library is loaded; the scan
  // leaves its ticket at zero and tags its status words per call)
  ScanCtl ctl;
  ctl.ticket = reinterpret_cast<unsigned *>(b + kScanOff);
  ctl.status = reinterpret_cast<unsigned long long *>(b + kScanOff + 256);
  ctl.tiles = kScanStatus;
  ctl.err = err;
  hpm_status s = radix_sort_pairs(k0, k1, v0, v1, n, 3 * max_depth, hist, ctl, st, nullptr);
  hist.p = nullptr;
  hist.cap = 0;
  if (s != HPM_OK) return s;
  if (k0 != d_keys) HPM_CUDA(cudaMemcpyAsync(d_keys, k0, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st));
  if (v0 != d_perm) HPM_CUDA(cudaMemcpyAsync(d_perm, v0, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st));
  int h_err = 0;
  HPM_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  HPM_CUDA(cudaStreamSynchronize(st));
  if (h_err & kErrTimeout) return HPM_ERR_TIMEOUT;
  return (h_err & kErrDomain) ? HPM_ERR_OUT_OF_DOMAIN : HPM_OK;
}
