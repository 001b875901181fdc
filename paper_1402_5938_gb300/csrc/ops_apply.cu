// Instantiation and launch of the FP32 operator-apply kernel (TMA-staged geometric factors).
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "dispatch.cuh"
#include "ops.cuh"
#include "pencil.cuh"

namespace hmg {

namespace {

// resident blocks per SM of (kernel, dynamic shared memory), queried once
int blocks_per_sm(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(kernel, threads, smem, dev);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int nb = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1) nb = 1;
  cache[key] = nb;
  return nb;
}

template <int DIM>
cudaError_t apply32_dim(const Mesh& m, const Basis1D& b, const float* x, float* y, const float* G, float alpha,
                        int* err, int variant, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    if constexpr (DIM == 3 && N <= kMaxNPlane) {
      if (variant == 6) return launch_plane<N, float>(m, b, x, y, G, nullptr, alpha, s);
    }
    if (variant >= 4)
      return launch_pencil<DIM, N, float>(m, b, x, y, G, nullptr, alpha, variant != 4, s);
    if constexpr (N <= kMaxNWarp32) {
      if (variant == 3) {  // warp-group form
        using W = Apply32wCfg<DIM, N>;
        const int wpb = 4;
        const size_t smem = (size_t)wpb * W::WARP_BYTES;
        auto kw = k_apply32w<DIM, N>;
        cudaError_t e = ensure_smem(kw, smem);
        if (e != cudaSuccess) return e;
        const long long ngroups = (m.nelem + W::EW - 1) / W::EW;
        if (ngroups == 0) return cudaSuccess;
        const long long grid = std::min<long long>((ngroups + wpb - 1) / wpb,
                                                   (long long)device_sm_count() * blocks_per_sm((const void*)kw, 32 * wpb, smem));
        kw<<<(unsigned)grid, 32 * wpb, smem, s>>>(x, y, G, m, make_tab<N, float>(b), alpha, ngroups);
        return counted(cudaGetLastError());
      }
    }
    constexpr int NP = Sh<DIM, N>::NP, NC = Sh<DIM, N>::NC;
    constexpr int NBUF = (DIM == 2 || NP <= 3200) ? 2 : 1;
    using C = Apply32Cfg<DIM, N, NBUF>;
    const size_t per = (size_t)(NBUF * NC + 1 + DIM) * NP * 4;
    // variant 0: ~64 KB of shared memory per block; 1: half the tile; 2: double the tile
    const size_t target = variant == 1 ? 32 * 1024 : (variant == 2 ? 128 * 1024 : 64 * 1024);
    int epb = (int)std::max<size_t>(1, target / per);
    const long long want = std::max(1LL, m.nelem / (2LL * device_sm_count()));
    if (epb > want) epb = (int)want;
    if (epb > 64) epb = 64;
    const size_t smem = C::smem(epb);
    auto kern = k_apply32<DIM, N, NBUF>;
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (m.nelem + epb - 1) / epb;
    if (ntiles == 0) return cudaSuccess;
    // one thread per line of a contraction phase (epb * N^(d-1) lines), rounded up to whole
    // warps; tiles with fewer lines keep 256 threads for their point-parallel phases
    constexpr int NL = Sh<DIM, N>::NL;
    const int lines = epb * NL;
    const int threads = lines >= 160 ? std::min(512, (lines + 31) / 32 * 32) : 256;
    const long long grid =
        std::min<long long>(ntiles, (long long)device_sm_count() * blocks_per_sm((const void*)kern, threads, smem));
    kern<<<(unsigned)grid, threads, smem, s>>>(x, y, G, m, make_tab<N, float>(b), alpha, epb, ntiles, err);
    return counted(cudaGetLastError());
  });
}

}  // namespace

cudaError_t launch_apply_f32(const Mesh& m, const Basis1D& b, const float* x, float* y,
                             const float* G, float alpha, int* err, cudaStream_t s, int variant) {
  return m.dim == 3 ? apply32_dim<3>(m, b, x, y, G, alpha, err, variant, s)
                    : apply32_dim<2>(m, b, x, y, G, alpha, err, variant, s);
}

}  // namespace hmg
