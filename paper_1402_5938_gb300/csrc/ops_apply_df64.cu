// The finest level's FP64 operator in double-float arithmetic (paper Sec. 2.3 matrix-free apply by
// sum factorization; the arithmetic is df64.cuh's): y += alpha A x with FP64 vectors, the FP64
// geometric factors split once into float pairs, and every contraction, pointwise product and
// accumulation in pairs of FP32 numbers. The pencil form of pencil.cuh carries it unchanged (one
// thread per element line, even/odd line products from order 4 on), factors read at their use.
#include "ops.cuh"
#include "pencil.cuh"

namespace hmg {

bool df64_supported(int dim, int n) { return n >= 2 && n <= kDf64MaxN && pencil64_fits(dim, n); }

namespace {
template <int DIM, int N>
cudaError_t apply_df64_n(const Mesh& m, const Basis1D& b, const double* x, double* y, const void* Gdf,
                         double alpha, cudaStream_t s) {
  return launch_pencil_gm<DIM, N, df64, 2, df64, double>(m, b, x, y, static_cast<const df64*>(Gdf), nullptr,
                                                        df64(alpha), s);
}
template <int DIM>
cudaError_t apply_df64_dim(const Mesh& m, const Basis1D& b, const double* x, double* y, const void* Gdf,
                           double alpha, cudaStream_t s) {
  switch (b.n) {
    case 2: return apply_df64_n<DIM, 2>(m, b, x, y, Gdf, alpha, s);
    case 3: return apply_df64_n<DIM, 3>(m, b, x, y, Gdf, alpha, s);
    case 4: return apply_df64_n<DIM, 4>(m, b, x, y, Gdf, alpha, s);
    case 5: return apply_df64_n<DIM, 5>(m, b, x, y, Gdf, alpha, s);
    case 6: return apply_df64_n<DIM, 6>(m, b, x, y, Gdf, alpha, s);
    case 7: return apply_df64_n<DIM, 7>(m, b, x, y, Gdf, alpha, s);
    case 8: return apply_df64_n<DIM, 8>(m, b, x, y, Gdf, alpha, s);
    case 9: return apply_df64_n<DIM, 9>(m, b, x, y, Gdf, alpha, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_split_df64(const double* __restrict__ G, float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const df64 v(G[i]);
    out[i] = make_float2(v.hi, v.lo);
  }
}
}  // namespace

cudaError_t launch_apply_df64(const Mesh& m, const Basis1D& b, const double* x, double* y, const void* Gdf,
                              double alpha, cudaStream_t s) {
  static_assert(kDf64MaxN == 9, "the dispatch above covers N = 2..9");
  return m.dim == 3 ? apply_df64_dim<3>(m, b, x, y, Gdf, alpha, s) : apply_df64_dim<2>(m, b, x, y, Gdf, alpha, s);
}

cudaError_t launch_split_df64(const double* G, void* Gdf, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long g = (n + 255) / 256;
  const long long cap = (long long)device_sm_count() * 16;
  if (g > cap) g = cap;
  k_split_df64<<<(unsigned)g, 256, 0, s>>>(G, static_cast<float2*>(Gdf), n);
  return counted(cudaGetLastError());
}

}  // namespace hmg
