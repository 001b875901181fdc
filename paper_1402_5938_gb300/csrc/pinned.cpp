// Process-wide pool of page-locked host blocks. Allocating page-locked memory is an implicit
// synchronization point of the device (commands of different streams cannot overlap across
// it), so the library takes its small pinned buffers (read-back scalars, residual histories,
// the server's staging vectors) from power-of-two size classes that are filled once and reused;
// blocks go back to their class, never to the system.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace hmg {

namespace {

constexpr int kClasses = 40;  // 64 B << k

int class_of(size_t bytes) {
  int k = 0;
  size_t c = 64;
  while (c < bytes && k + 1 < kClasses) {
    c <<= 1;
    ++k;
  }
  return k;
}

std::mutex& pool_mu() {
  static std::mutex m;
  return m;
}
std::vector<void*>* free_lists() {
  static std::vector<void*> lists[kClasses];
  return lists;
}

}  // namespace

void* pinned_alloc(size_t bytes) {
  const int k = class_of(bytes == 0 ? 1 : bytes);
  {
    std::lock_guard<std::mutex> lk(pool_mu());
    auto& fl = free_lists()[k];
    if (!fl.empty()) {
      void* p = fl.back();
      fl.pop_back();
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, (size_t)64 << k) != cudaSuccess) return nullptr;
  return p;
}

void pinned_free(void* p, size_t bytes) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(pool_mu());
  free_lists()[class_of(bytes == 0 ? 1 : bytes)].push_back(p);
}

}  // namespace hmg

namespace hmg {

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  static std::mutex mu;
  static bool configured[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(mu);
    if (!configured[dev]) {
      // keep freed blocks in the pool for later problems instead of unmapping them at the
      // next synchronization (this process's pool only)
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
      configured[dev] = true;
    }
  }
  return cudaMallocAsync(p, bytes == 0 ? 16 : bytes, s);
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

}  // namespace hmg
