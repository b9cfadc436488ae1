// Block counts and means with no allocation at all.
//
// Some callers cannot allocate device memory while they run: a serving
// process that hands all of its device memory to its own pool up front, or
// a real-time loop whose memory footprint is fixed before it starts. For
// them bsvd_block_means_noalloc runs the partition's counting and mean
// kernels with their scratch (per-block sums, block bounds, the largest
// |rating| and the error word) in one file-scope __device__ array instead
// of context-owned buffers. The caller passes device inputs and outputs.
//
// The array holds at most kNoAllocMaxBlocks blocks and kNoAllocMaxSide + 1
// bounds per side; larger grids are rejected. Every GPU that loads the
// library keeps the array until the process exits. All calls share it and
// it keeps the last call's contents, so each call clears what must start
// at zero, and calls that overlap on the GPU (different streams or
// threads, or a second call queued before the first finishes) race on it.
#include <mutex>

#include "bsvd.h"
#include "kernels.h"

using namespace bsvd;

namespace {

constexpr int kNoAllocMaxBlocks = 4096;
constexpr int kNoAllocMaxSide = 4096;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  long long sums[kNoAllocMaxBlocks];            // fixed-point rating sums
  int64_t row_bounds[kNoAllocMaxSide + 1];
  int64_t col_bounds[kNoAllocMaxSide + 1];
  unsigned int maxabs_bits;                     // bits of max |x|
  int32_t err;                                  // kErr* flags
};

// The scratch itself. In host code this name is only a stand-in for the
// device symbol; kernels get its device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char
    g_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_setup_mutex;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device (set up once per
// device, with that device current). The address stays valid while the
// device's primary context lives; after cudaDeviceReset the library must
// not be used again in this process.
cudaError_t scratch_address(NoAllocScratch **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<NoAllocScratch *>(ptr);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

__global__ void k_equal_bounds(int64_t *bounds, int32_t parts, int64_t total,
                               int64_t size) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= parts;
       j += gridDim.x * blockDim.x) {
    const int64_t v = (int64_t)j * size;
    bounds[j] = v < total ? v : total;
  }
}

// True for managed memory and for device memory of the current device. A
// device pointer of another GPU is refused: the kernels would reach it
// through a peer mapping that may not exist.
bool on_device(const void *ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  if (a.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.device == dev;
}

}  // namespace

extern "C" bsvd_status bsvd_block_means_noalloc(
    int64_t m, int64_t n, int64_t nnz, const int32_t *u, const int32_t *i,
    const float *x, int32_t p, int32_t q, int64_t *counts, float *mu,
    void *stream) {
  if (m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || nnz < 0 ||
      p < 1 || q < 1 || p > m || q > n)
    return BSVD_EINVAL;
  if (p > kNoAllocMaxSide || q > kNoAllocMaxSide ||
      (int64_t)p * q > kNoAllocMaxBlocks)
    return BSVD_EINVAL;
  if (!counts || !mu || !on_device(counts) || !on_device(mu))
    return BSVD_EINVAL;
  if (nnz > 0 && (!u || !i || !x || !on_device(u) || !on_device(i) ||
                  !on_device(x)))
    return BSVD_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  NoAllocScratch *sc = nullptr;
  if (scratch_address(&sc) != cudaSuccess) {
    cudaGetLastError();
    return BSVD_ECUDA;
  }
  const int32_t nb = p * q;
  const int64_t br = (m + p - 1) / p, bc = (n + q - 1) / q;
  cudaError_t e = cudaSuccess;
  // clear what the kernels accumulate into
  if (e == cudaSuccess) e = cudaMemsetAsync(sc->sums, 0, sizeof(long long) * nb, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&sc->maxabs_bits, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(&sc->err, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * nb, st);
  if (e == cudaSuccess) {
    k_equal_bounds<<<(p + 256) / 256, 256, 0, st>>>(sc->row_bounds, p, m, br);
    k_equal_bounds<<<(q + 256) / 256, 256, 0, st>>>(sc->col_bounds, q, n, bc);
    e = cudaGetLastError();
  }
  GridDesc g{};
  g.m = m; g.n = n; g.p = p; g.q = q;
  g.equal_rows = 1; g.equal_cols = 1;
  g.br = br; g.bc = bc;
  g.row_bounds = sc->row_bounds;
  g.col_bounds = sc->col_bounds;
  g.row_perm = nullptr;
  g.col_perm = nullptr;
  if (e == cudaSuccess)
    e = launch_count(g, nnz, u, i, x, nb,
                     reinterpret_cast<unsigned long long *>(counts), sc->sums,
                     &sc->maxabs_bits, &sc->err, st);
  if (e == cudaSuccess)
    e = launch_means(nb, reinterpret_cast<unsigned long long *>(counts),
                     sc->sums, &sc->maxabs_bits, mu, &sc->err, st);
  int32_t h_err = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_err, &sc->err, sizeof h_err, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BSVD_ECUDA;
  }
  return h_err ? BSVD_EINVAL : BSVD_OK;
}
