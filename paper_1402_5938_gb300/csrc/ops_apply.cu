// Instantiation and launch of the operator-apply kernels (FP64 and FP32).
#include <algorithm>

#include "dispatch.cuh"
#include "ops.cuh"

namespace hmg {

namespace {

template <int DIM, typename T>
cudaError_t apply_dim(const Mesh& m, const Basis1D& b, const T* x, T* y, const T* G, T alpha,
                      cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    constexpr int NP = Sh<DIM, N>::NP;
    const size_t per = (size_t)(1 + DIM) * NP * sizeof(T);
    // shared-memory cap, then small enough tiles for >= 4 blocks per SM on the 152 SMs
    int epb = epb_for(per);
    const long long want = std::max(1LL, m.nelem / (152LL * 4));
    if (epb > want) epb = (int)want;
    const size_t smem = per * epb;
    auto kern = k_apply<DIM, N, T>;
    cudaError_t e = ensure_smem(kern, smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + epb - 1) / epb;
    if (blocks == 0) return cudaSuccess;
    kern<<<(unsigned)blocks, 256, smem, s>>>(x, y, G, m, make_tab<N, T>(b), alpha, epb);
    return counted(cudaGetLastError());
  });
}

}  // namespace

template <int DIM>
cudaError_t apply64_dim(const Mesh& m, const Basis1D& b, const double* x, double* y, const double* G,
                        double alpha, cudaStream_t s) {
  return dispatch_n(b.n, [&](auto nc) -> cudaError_t {
    constexpr int N = decltype(nc)::value;
    using C = Apply64Cfg<DIM, N>;
    auto kern = k_apply64<DIM, N>;
    cudaError_t e = ensure_smem(kern, C::smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (m.nelem + C::NEG - 1) / C::NEG;
    if (blocks == 0) return cudaSuccess;
    kern<<<(unsigned)blocks, C::GT, C::smem, s>>>(x, y, G, m, make_tab<N, double>(b), alpha);
    return counted(cudaGetLastError());
  });
}

cudaError_t launch_apply_f64(const Mesh& m, const Basis1D& b, const double* x, double* y,
                             const double* G, double alpha, cudaStream_t s) {
  return m.dim == 3 ? apply64_dim<3>(m, b, x, y, G, alpha, s) : apply64_dim<2>(m, b, x, y, G, alpha, s);
}

cudaError_t launch_apply_f32(const Mesh& m, const Basis1D& b, const float* x, float* y,
                             const float* G, float alpha, cudaStream_t s) {
  return m.dim == 3 ? apply_dim<3, float>(m, b, x, y, G, alpha, s)
                    : apply_dim<2, float>(m, b, x, y, G, alpha, s);
}

}  // namespace hmg
