// Instantiation and launch of the FP16 / BF16 tensor-core apply (orders p <= 7) and of the
// packing of its geometric factors.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "dispatch.cuh"
#include "element16.cuh"
#include "ops.cuh"
#include "pencil.cuh"

namespace hmg {

namespace {

int resident16(const void* kernel, int threads, size_t smem) {
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

Tab16 make_tab16(const Basis1D& b) {
  Tab16 t{};
  for (int i = 0; i < b.n * b.n; ++i) {
    t.B[i] = (float)b.B[i];
    t.Bd[i] = (float)b.Bd[i];
  }
  return t;
}

template <int DIM, int N, typename T, int HALF>
cudaError_t apply16_launch(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G16,
                           const float* gsc, float alpha, int* err, int wpb, cudaStream_t s) {
  using C = Apply16Cfg<DIM, N, HALF>;
  const size_t smem = C::smem(wpb);
  auto kern = k_apply16<DIM, N, T, HALF>;
  cudaError_t e = ensure_smem(kern, smem);
  if (e != cudaSuccess) return e;
  const long long ngroups = (m.nelem + C::EW - 1) / C::EW;
  if (ngroups == 0) return cudaSuccess;
  const long long blocks = (ngroups + wpb - 1) / wpb;
  const long long grid =
      std::min<long long>(blocks, (long long)device_sm_count() * resident16((const void*)kern, 32 * wpb, smem));
  kern<<<(unsigned)grid, 32 * wpb, smem, s>>>(x, y, static_cast<const T*>(G16), gsc, m, make_tab16(b), alpha,
                                              ngroups, err);
  return counted(cudaGetLastError());
}

template <int DIM, typename T>
cudaError_t apply16_dim(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G16,
                        const float* gsc, float alpha, int* err, int variant, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    // variants 4, 5: the pencil form with 16-bit factors and FP32 arithmetic (every order; 5 keeps
    // the factors in registers from the start); orders above the tensor-core kernel's take 4
    if constexpr (DIM == 3 && N <= kMaxNPlane) {
      if (variant == 6) return launch_plane<N, T>(m, b, x, y, static_cast<const T*>(G16), gsc, alpha, s);
    }
    if (variant >= 4 || N > kMaxN16)
      return launch_pencil<DIM, N, T>(m, b, x, y, static_cast<const T*>(G16), gsc, alpha, variant >= 5, s);
    if constexpr (N > kMaxN16) {
      return cudaErrorInvalidValue;
    } else {
      // variant 0: 4 warps per block, 1: 2 warps, 2: 8 warps, 3: 4 warps with half-size groups
      if (variant == 3) return apply16_launch<DIM, N, T, 1>(m, b, x, y, G16, gsc, alpha, err, 4, s);
      const int wpb = variant == 1 ? 2 : (variant == 2 ? 8 : 4);
      return apply16_launch<DIM, N, T, 0>(m, b, x, y, G16, gsc, alpha, err, wpb, s);
    }
  });
}

}  // namespace

cudaError_t launch_apply_lowp(const Mesh& m, const Basis1D& b, const float* x, float* y, const void* G16,
                              const float* gsc, float alpha, int prec, int* err, cudaStream_t s, int variant) {
  if (prec == HMG_PREC_FP16)
    return m.dim == 3 ? apply16_dim<3, __half>(m, b, x, y, G16, gsc, alpha, err, variant, s)
                      : apply16_dim<2, __half>(m, b, x, y, G16, gsc, alpha, err, variant, s);
  if (prec == HMG_PREC_BF16)
    return m.dim == 3 ? apply16_dim<3, __nv_bfloat16>(m, b, x, y, G16, gsc, alpha, err, variant, s)
                      : apply16_dim<2, __nv_bfloat16>(m, b, x, y, G16, gsc, alpha, err, variant, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_pack_g16(const double* G, void* G16, float* gsc, long long nelem, int nc, int np, int dim,
                            int prec, cudaStream_t s) {
  if (nelem == 0) return cudaSuccess;
  const int pm = dim == 3;  // the 3D kernel reads a point's six factors as three 32-bit words
  if (prec == HMG_PREC_FP16)
    k_pack_g16<__half><<<(unsigned)nelem, 128, 0, s>>>(G, static_cast<__half*>(G16), gsc, nelem, nc, np, pm);
  else if (prec == HMG_PREC_BF16)
    k_pack_g16<__nv_bfloat16><<<(unsigned)nelem, 128, 0, s>>>(G, static_cast<__nv_bfloat16*>(G16), nullptr,
                                                             nelem, nc, np, pm);
  else
    return cudaErrorInvalidValue;
  return counted(cudaGetLastError());
}

}  // namespace hmg
