// Instantiation and launch of the FP64 operator apply: the point-parallel kernel (all orders, four
// block shapes), stored element matrices (orders 1-2), and the pencil form in FP64 arithmetic with
// even/odd line products (pencil.cuh).
#include <algorithm>

#include "dispatch.cuh"
#include "ops.cuh"
#include "pencil.cuh"

namespace hmg {

namespace {

template <int DIM, int N, int V>
cudaError_t apply64_variant(const Mesh& m, const Basis1D& b, const double* x, double* y, const double* G,
                            double alpha, int* err, cudaStream_t s) {
  using C = Apply64Cfg<DIM, N, V>;
  auto kern = k_apply64<DIM, N, V>;
  cudaError_t e = ensure_smem(kern, C::smem);
  if (e != cudaSuccess) return e;
  const long long blocks = (m.nelem + C::NEG - 1) / C::NEG;
  if (blocks == 0) return cudaSuccess;
  kern<<<(unsigned)blocks, C::GT, C::smem, s>>>(x, y, G, m, make_tab<N, double>(b), alpha, alpha_mode(alpha), err);
  return counted(cudaGetLastError());
}

template <int DIM>
cudaError_t apply64_dim(const Mesh& m, const Basis1D& b, const double* x, double* y, const double* G,
                        double alpha, int* err, int variant, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    switch (variant) {
      case 1: return apply64_variant<DIM, N, 1>(m, b, x, y, G, alpha, err, s);
      case 2: return apply64_variant<DIM, N, 2>(m, b, x, y, G, alpha, err, s);
      case 3: return apply64_variant<DIM, N, 3>(m, b, x, y, G, alpha, err, s);
      default: return apply64_variant<DIM, N, 0>(m, b, x, y, G, alpha, err, s);
    }
  });
}

}  // namespace

template <int DIM>
cudaError_t apply_dense64_dim(const Mesh& m, const Basis1D& b, const double* x, double* y, const double* Ke,
                              double alpha, cudaStream_t s) {
  if (b.n > kMaxNDense) return cudaErrorInvalidValue;
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    if constexpr (N > kMaxNDense) {
      return cudaErrorInvalidValue;
    } else {
      constexpr int EPB = 256 / Sh<DIM, N>::NP;
      const long long groups = (m.nelem + EPB - 1) / EPB;
      if (groups == 0) return cudaSuccess;
      const unsigned grid = (unsigned)std::min<long long>(groups, (long long)device_sm_count() * 8);
      k_apply_dense64<DIM, N><<<grid, 256, 0, s>>>(x, y, Ke, m, alpha);
      return counted(cudaGetLastError());
    }
  });
}

bool pencil64_fits(int dim, int n) {
  const PencilShape sh = pencil_shape(dim, n);
  const size_t bytes = (size_t)(dim == 3 ? 4 : 3) * sh.epb * sh.ep * sizeof(double);
  return bytes <= 227 * 1024;
}

template <int DIM>
cudaError_t apply_pencil64_dim(const Mesh& m, const Basis1D& b, const double* x, double* y, const double* G,
                               double alpha, int variant, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    if constexpr (N <= kPencil64AheadMaxN) {
      if (variant == kApply64PencilAhead)
        return launch_pencil_gm<DIM, N, double, 0, double>(m, b, x, y, G, nullptr, alpha, s);
    }
    return launch_pencil_gm<DIM, N, double, 2, double>(m, b, x, y, G, nullptr, alpha, s);
  });
}

cudaError_t launch_apply_f64(const Mesh& m, const Basis1D& b, const double* x, double* y,
                             const double* G, double alpha, int* err, cudaStream_t s, int variant,
                             const double* Ke, const void* Gdf) {
  if (variant == kApply64Df) {
    if (Gdf == nullptr || !df64_supported(m.dim, b.n)) return cudaErrorInvalidValue;
    return launch_apply_df64(m, b, x, y, Gdf, alpha, s);
  }
  if (variant == kApply64Pencil || variant == kApply64PencilAhead) {
    if (!pencil64_fits(m.dim, b.n)) return cudaErrorInvalidValue;
    return m.dim == 3 ? apply_pencil64_dim<3>(m, b, x, y, G, alpha, variant, s)
                      : apply_pencil64_dim<2>(m, b, x, y, G, alpha, variant, s);
  }
  if (variant == kApply64Dense && Ke != nullptr)
    return m.dim == 3 ? apply_dense64_dim<3>(m, b, x, y, Ke, alpha, s) : apply_dense64_dim<2>(m, b, x, y, Ke, alpha, s);
  return m.dim == 3 ? apply64_dim<3>(m, b, x, y, G, alpha, err, variant, s)
                    : apply64_dim<2>(m, b, x, y, G, alpha, err, variant, s);
}

}  // namespace hmg
